// pat_p2_f32.cu -- the power-of-two persistent kernel instantiated for float fields (any size; the
// 256^2 and 512^2 grids run the fixed-size instances of pat_p2_f32_n256.cu / pat_p2_f32_n512.cu).
#include "pat_persist2.cuh"

namespace pat {

template <>
cudaError_t p2_launch<float>(bool adjoint, const cudaLaunchConfig_t* lc, const DevPlan<float>& P, const PersistCfg& C,
                          unsigned* gbar) {
    switch (p2_sq_lg(P.fx.lgn, P.fy.lgn, P.fixed_len)) {
        case 8: return p2_launch_f32_sq<8>(adjoint, lc, P, C, gbar);
        case 9: return p2_launch_f32_sq<9>(adjoint, lc, P, C, gbar);
        default: break;
    }
    if (adjoint) return cudaLaunchKernelEx(lc, k_persist2<float, true>, P, C, gbar);
    return cudaLaunchKernelEx(lc, k_persist2<float, false>, P, C, gbar);
}

template <> const void* p2_kernel<float>(bool adjoint, int lgx, int lgy, int fixed_len) {
    switch (p2_sq_lg(lgx, lgy, fixed_len)) {
        case 8: return p2_kernel_f32_sq<8>(adjoint);
        case 9: return p2_kernel_f32_sq<9>(adjoint);
        default: break;
    }
    return adjoint ? (const void*)k_persist2<float, true> : (const void*)k_persist2<float, false>;
}

}  // namespace pat
