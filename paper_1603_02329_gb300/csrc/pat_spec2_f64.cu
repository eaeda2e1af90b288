// pat_spec2_f64.cu -- the power-of-two spectral kernels instantiated for double fields.
#include "pat_spec2.cuh"

namespace pat {

template <>
cudaError_t spec2_launch<double>(const cudaLaunchConfig_t* lc, int D, int mode, const DevPlan<double>& P, int W, int lgW,
                             int lax, int F) {
    switch (D * 8 + mode) {
        case 2 * 8 + SPEC_PLAIN_FWD: return cudaLaunchKernelEx(lc, k_spec2<double, 2, SPEC_PLAIN_FWD>, P, W, lgW, lax, F);
        case 2 * 8 + SPEC_PLAIN_INV: return cudaLaunchKernelEx(lc, k_spec2<double, 2, SPEC_PLAIN_INV>, P, W, lgW, lax, F);
        case 2 * 8 + SPEC_GRAD: return cudaLaunchKernelEx(lc, k_spec2<double, 2, SPEC_GRAD>, P, W, lgW, lax, F);
        case 2 * 8 + SPEC_DIV: return cudaLaunchKernelEx(lc, k_spec2<double, 2, SPEC_DIV>, P, W, lgW, lax, F);
        case 2 * 8 + SPEC_ABS: return cudaLaunchKernelEx(lc, k_spec2<double, 2, SPEC_ABS>, P, W, lgW, lax, F);
        case 2 * 8 + SPEC_DIVT: return cudaLaunchKernelEx(lc, k_spec2<double, 2, SPEC_DIVT>, P, W, lgW, lax, F);
        case 2 * 8 + SPEC_GRADT: return cudaLaunchKernelEx(lc, k_spec2<double, 2, SPEC_GRADT>, P, W, lgW, lax, F);
        case 3 * 8 + SPEC_PLAIN_FWD: return cudaLaunchKernelEx(lc, k_spec2<double, 3, SPEC_PLAIN_FWD>, P, W, lgW, lax, F);
        case 3 * 8 + SPEC_PLAIN_INV: return cudaLaunchKernelEx(lc, k_spec2<double, 3, SPEC_PLAIN_INV>, P, W, lgW, lax, F);
        case 3 * 8 + SPEC_GRAD: return cudaLaunchKernelEx(lc, k_spec2<double, 3, SPEC_GRAD>, P, W, lgW, lax, F);
        case 3 * 8 + SPEC_DIV: return cudaLaunchKernelEx(lc, k_spec2<double, 3, SPEC_DIV>, P, W, lgW, lax, F);
        case 3 * 8 + SPEC_ABS: return cudaLaunchKernelEx(lc, k_spec2<double, 3, SPEC_ABS>, P, W, lgW, lax, F);
        case 3 * 8 + SPEC_DIVT: return cudaLaunchKernelEx(lc, k_spec2<double, 3, SPEC_DIVT>, P, W, lgW, lax, F);
        case 3 * 8 + SPEC_GRADT: return cudaLaunchKernelEx(lc, k_spec2<double, 3, SPEC_GRADT>, P, W, lgW, lax, F);
        default: return cudaErrorInvalidValue;
    }
}

template <> cudaError_t spec2_set_attrs<double>(int bytes) {
    const void* ks[] = {
        (const void*)k_spec2<double, 2, SPEC_PLAIN_FWD>,
        (const void*)k_spec2<double, 2, SPEC_PLAIN_INV>,
        (const void*)k_spec2<double, 2, SPEC_GRAD>,
        (const void*)k_spec2<double, 2, SPEC_DIV>,
        (const void*)k_spec2<double, 2, SPEC_ABS>,
        (const void*)k_spec2<double, 2, SPEC_DIVT>,
        (const void*)k_spec2<double, 2, SPEC_GRADT>,
        (const void*)k_spec2<double, 3, SPEC_PLAIN_FWD>,
        (const void*)k_spec2<double, 3, SPEC_PLAIN_INV>,
        (const void*)k_spec2<double, 3, SPEC_GRAD>,
        (const void*)k_spec2<double, 3, SPEC_DIV>,
        (const void*)k_spec2<double, 3, SPEC_ABS>,
        (const void*)k_spec2<double, 3, SPEC_DIVT>,
        (const void*)k_spec2<double, 3, SPEC_GRADT>,
    };
    for (const void* k : ks) {
        cudaError_t e = set_dyn_smem(k, bytes);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace pat
