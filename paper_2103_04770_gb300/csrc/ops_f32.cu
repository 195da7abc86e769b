// FP32 instantiation of the spectral and Krylov operators (mixed precision).
#include "ops.cuh"
namespace rvk { template struct Ops<float>; }
