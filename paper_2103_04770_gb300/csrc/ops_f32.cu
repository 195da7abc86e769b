// FP32 instantiation of the spectral and Krylov operators (mixed precision).
#include "ops.cuh"
namespace rvk {
template struct Ops<float>;
template void Ops<float>::xinv_residual<float>(const Geo&, const Tables<float>&, const LaunchCfg&,
                                               cudaStream_t, const C2<float>*, float*, const double*,
                                               const double*, const double*, double*,
                                               const float*, const double*);
}  // namespace rvk
