// pat_p2_f64.cu -- the power-of-two persistent kernel instantiated for double fields.
#include "pat_persist2.cuh"

namespace pat {

template <>
cudaError_t p2_launch<double>(bool adjoint, const cudaLaunchConfig_t* lc, const DevPlan<double>& P, const PersistCfg& C,
                          unsigned* gbar) {
    if (adjoint) return cudaLaunchKernelEx(lc, k_persist2<double, true>, P, C, gbar);
    return cudaLaunchKernelEx(lc, k_persist2<double, false>, P, C, gbar);
}

template <> const void* p2_kernel<double>(bool adjoint, int, int, int) {
    return adjoint ? (const void*)k_persist2<double, true> : (const void*)k_persist2<double, false>;
}

}  // namespace pat
