// pat_p2_f32_n512.cu -- the power-of-two persistent kernel compiled for 512 x 512 grids, float fields.
#include "pat_persist2.cuh"

namespace pat {

template <>
cudaError_t p2_launch_f32_sq<9>(bool adjoint, const cudaLaunchConfig_t* lc, const DevPlan<float>& P, const PersistCfg& C,
                                 unsigned* gbar) {
    if (adjoint) return cudaLaunchKernelEx(lc, k_persist2<float, true, 9, 9>, P, C, gbar);
    return cudaLaunchKernelEx(lc, k_persist2<float, false, 9, 9>, P, C, gbar);
}

template <> const void* p2_kernel_f32_sq<9>(bool adjoint) {
    return adjoint ? (const void*)k_persist2<float, true, 9, 9> : (const void*)k_persist2<float, false, 9, 9>;
}

}  // namespace pat
