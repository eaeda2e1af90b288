// pat_spec2_f32.cu -- the power-of-two spectral kernels instantiated for float fields (any length; 3-D
// lines of 64, 128 and 256 points run the fixed-length instances of pat_spec2_f32_n*.cu).
#include "pat_spec2.cuh"

namespace pat {

template <>
cudaError_t spec2_launch<float>(const cudaLaunchConfig_t* lc, int D, int mode, const DevPlan<float>& P, int W, int lgW,
                             int lax, int F) {
    if (D == 3) {
        switch (p2_3d_lg(lax == 1 ? P.fy.lgn : P.fz.lgn, P.fixed_len)) {
            case 6: return spec2_launch_f32_3d<6>(lc, mode, P, W, lgW, lax, F);
            case 7: return spec2_launch_f32_3d<7>(lc, mode, P, W, lgW, lax, F);
            case 8: return spec2_launch_f32_3d<8>(lc, mode, P, W, lgW, lax, F);
            default: break;
        }
    }
    switch (D * 8 + mode) {
        case 2 * 8 + SPEC_PLAIN_FWD: return cudaLaunchKernelEx(lc, k_spec2<float, 2, SPEC_PLAIN_FWD>, P, W, lgW, lax, F);
        case 2 * 8 + SPEC_PLAIN_INV: return cudaLaunchKernelEx(lc, k_spec2<float, 2, SPEC_PLAIN_INV>, P, W, lgW, lax, F);
        case 2 * 8 + SPEC_GRAD: return cudaLaunchKernelEx(lc, k_spec2<float, 2, SPEC_GRAD>, P, W, lgW, lax, F);
        case 2 * 8 + SPEC_DIV: return cudaLaunchKernelEx(lc, k_spec2<float, 2, SPEC_DIV>, P, W, lgW, lax, F);
        case 2 * 8 + SPEC_ABS: return cudaLaunchKernelEx(lc, k_spec2<float, 2, SPEC_ABS>, P, W, lgW, lax, F);
        case 2 * 8 + SPEC_DIVT: return cudaLaunchKernelEx(lc, k_spec2<float, 2, SPEC_DIVT>, P, W, lgW, lax, F);
        case 2 * 8 + SPEC_GRADT: return cudaLaunchKernelEx(lc, k_spec2<float, 2, SPEC_GRADT>, P, W, lgW, lax, F);
        case 3 * 8 + SPEC_PLAIN_FWD: return cudaLaunchKernelEx(lc, k_spec2<float, 3, SPEC_PLAIN_FWD>, P, W, lgW, lax, F);
        case 3 * 8 + SPEC_PLAIN_INV: return cudaLaunchKernelEx(lc, k_spec2<float, 3, SPEC_PLAIN_INV>, P, W, lgW, lax, F);
        case 3 * 8 + SPEC_GRAD: return cudaLaunchKernelEx(lc, k_spec2<float, 3, SPEC_GRAD>, P, W, lgW, lax, F);
        case 3 * 8 + SPEC_DIV: return cudaLaunchKernelEx(lc, k_spec2<float, 3, SPEC_DIV>, P, W, lgW, lax, F);
        case 3 * 8 + SPEC_ABS: return cudaLaunchKernelEx(lc, k_spec2<float, 3, SPEC_ABS>, P, W, lgW, lax, F);
        case 3 * 8 + SPEC_DIVT: return cudaLaunchKernelEx(lc, k_spec2<float, 3, SPEC_DIVT>, P, W, lgW, lax, F);
        case 3 * 8 + SPEC_GRADT: return cudaLaunchKernelEx(lc, k_spec2<float, 3, SPEC_GRADT>, P, W, lgW, lax, F);
        default: return cudaErrorInvalidValue;
    }
}

template <> cudaError_t spec2_set_attrs<float>(int bytes) {
    const void* ks[] = {
        (const void*)k_spec2<float, 2, SPEC_PLAIN_FWD>,
        (const void*)k_spec2<float, 2, SPEC_PLAIN_INV>,
        (const void*)k_spec2<float, 2, SPEC_GRAD>,
        (const void*)k_spec2<float, 2, SPEC_DIV>,
        (const void*)k_spec2<float, 2, SPEC_ABS>,
        (const void*)k_spec2<float, 2, SPEC_DIVT>,
        (const void*)k_spec2<float, 2, SPEC_GRADT>,
        (const void*)k_spec2<float, 3, SPEC_PLAIN_FWD>,
        (const void*)k_spec2<float, 3, SPEC_PLAIN_INV>,
        (const void*)k_spec2<float, 3, SPEC_GRAD>,
        (const void*)k_spec2<float, 3, SPEC_DIV>,
        (const void*)k_spec2<float, 3, SPEC_ABS>,
        (const void*)k_spec2<float, 3, SPEC_DIVT>,
        (const void*)k_spec2<float, 3, SPEC_GRADT>,
    };
    for (const void* k : ks) {
        cudaError_t e = set_dyn_smem(k, bytes);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = spec2_set_attrs_f32_3d<6>(bytes);
    if (e == cudaSuccess) e = spec2_set_attrs_f32_3d<7>(bytes);
    if (e == cudaSuccess) e = spec2_set_attrs_f32_3d<8>(bytes);
    return e;
}

}  // namespace pat
