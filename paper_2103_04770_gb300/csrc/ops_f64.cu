// FP64 instantiation of the spectral and Krylov operators (the FP64 form,
// and the FP64 Newton residual of the mixed form, which stores b in FP32).
#include "ops.cuh"
namespace rvk {
template struct Ops<double>;
template void Ops<double>::xinv_residual<double>(const Geo&, const Tables<double>&, const LaunchCfg&,
                                                 cudaStream_t, const C2<double>*, double*, const double*,
                                                 const double*, const double*, double*, const double*,
                                                 const double*);
template void Ops<double>::xinv_residual<float>(const Geo&, const Tables<double>&, const LaunchCfg&,
                                                cudaStream_t, const C2<double>*, float*, const double*,
                                                const double*, const double*, double*, const float*,
                                                const double*);
}  // namespace rvk
