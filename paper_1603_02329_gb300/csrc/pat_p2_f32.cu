// pat_p2_f32.cu -- the power-of-two persistent kernel instantiated for float fields.
#include "pat_persist2.cuh"

namespace pat {

template <>
cudaError_t p2_launch<float>(bool adjoint, const cudaLaunchConfig_t* lc, const DevPlan<float>& P, const PersistCfg& C,
                          unsigned* gbar) {
    if (adjoint) return cudaLaunchKernelEx(lc, k_persist2<float, true>, P, C, gbar);
    return cudaLaunchKernelEx(lc, k_persist2<float, false>, P, C, gbar);
}

template <> const void* p2_kernel<float>(bool adjoint) {
    return adjoint ? (const void*)k_persist2<float, true> : (const void*)k_persist2<float, false>;
}

}  // namespace pat
