// pat_spec2_f32_n64.cu -- the 3-D power-of-two spectral kernels compiled for lines of 64 points,
// float fields.
#include "pat_spec2.cuh"

namespace pat {

template <>
cudaError_t spec2_launch_f32_3d<6>(const cudaLaunchConfig_t* lc, int mode, const DevPlan<float>& P, int W, int lgW,
                                    int lax, int F) {
    switch (mode) {
        case SPEC_PLAIN_FWD: return cudaLaunchKernelEx(lc, k_spec2<float, 3, SPEC_PLAIN_FWD, 6>, P, W, lgW, lax, F);
        case SPEC_PLAIN_INV: return cudaLaunchKernelEx(lc, k_spec2<float, 3, SPEC_PLAIN_INV, 6>, P, W, lgW, lax, F);
        case SPEC_GRAD: return cudaLaunchKernelEx(lc, k_spec2<float, 3, SPEC_GRAD, 6>, P, W, lgW, lax, F);
        case SPEC_DIV: return cudaLaunchKernelEx(lc, k_spec2<float, 3, SPEC_DIV, 6>, P, W, lgW, lax, F);
        case SPEC_ABS: return cudaLaunchKernelEx(lc, k_spec2<float, 3, SPEC_ABS, 6>, P, W, lgW, lax, F);
        case SPEC_DIVT: return cudaLaunchKernelEx(lc, k_spec2<float, 3, SPEC_DIVT, 6>, P, W, lgW, lax, F);
        case SPEC_GRADT: return cudaLaunchKernelEx(lc, k_spec2<float, 3, SPEC_GRADT, 6>, P, W, lgW, lax, F);
        default: return cudaErrorInvalidValue;
    }
}

template <> cudaError_t spec2_set_attrs_f32_3d<6>(int bytes) {
    const void* ks[] = {
        (const void*)k_spec2<float, 3, SPEC_PLAIN_FWD, 6>,
        (const void*)k_spec2<float, 3, SPEC_PLAIN_INV, 6>,
        (const void*)k_spec2<float, 3, SPEC_GRAD, 6>,
        (const void*)k_spec2<float, 3, SPEC_DIV, 6>,
        (const void*)k_spec2<float, 3, SPEC_ABS, 6>,
        (const void*)k_spec2<float, 3, SPEC_DIVT, 6>,
        (const void*)k_spec2<float, 3, SPEC_GRADT, 6>,
    };
    for (const void* k : ks) {
        cudaError_t e = set_dyn_smem(k, bytes);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace pat
