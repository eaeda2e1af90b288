// pat_p2_f32_n256.cu -- the power-of-two persistent kernel compiled for 256 x 256 grids, float fields.
#include "pat_persist2.cuh"

namespace pat {

template <>
cudaError_t p2_launch_f32_sq<8>(bool adjoint, const cudaLaunchConfig_t* lc, const DevPlan<float>& P, const PersistCfg& C,
                                 unsigned* gbar) {
    if (adjoint) return cudaLaunchKernelEx(lc, k_persist2<float, true, 8, 8>, P, C, gbar);
    return cudaLaunchKernelEx(lc, k_persist2<float, false, 8, 8>, P, C, gbar);
}

template <> const void* p2_kernel_f32_sq<8>(bool adjoint) {
    return adjoint ? (const void*)k_persist2<float, true, 8, 8> : (const void*)k_persist2<float, false, 8, 8>;
}

}  // namespace pat
