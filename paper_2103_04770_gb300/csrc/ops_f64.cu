// FP64 instantiation of the spectral and Krylov operators.
#include "ops.cuh"
namespace rvk { template struct Ops<double>; }
