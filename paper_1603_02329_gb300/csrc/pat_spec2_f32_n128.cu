// pat_spec2_f32_n128.cu -- the 3-D power-of-two spectral kernels compiled for lines of 128 points,
// float fields: the two-stage schedule (k_spec16, radices 8 and 16) for the plain transforms, the
// fixed schedule of k_spec2 for the fused multiply passes; DevPlan::spec16 selects (3: the two-stage
// schedule also for the multiply passes whose fields are independent, DIV, DIVT and ABS).
#include "pat_spec16.cuh"

namespace pat {

template <>
cudaError_t spec2_launch_f32_3d<7>(const cudaLaunchConfig_t* lc, int mode, const DevPlan<float>& P, int W, int lgW,
                                    int lax, int F) {
    const bool plain = (mode == SPEC_PLAIN_FWD || mode == SPEC_PLAIN_INV);
    const bool fieldwise = (mode == SPEC_DIV || mode == SPEC_DIVT || mode == SPEC_ABS);
    if (P.stw16[lax] && (P.spec16 == 2 || (P.spec16 >= 1 && plain) || (P.spec16 == 3 && fieldwise))) {
        switch (mode) {
            case SPEC_PLAIN_FWD: return cudaLaunchKernelEx(lc, k_spec16<float, 3, SPEC_PLAIN_FWD, 7>, P, W, lgW, lax, F);
            case SPEC_PLAIN_INV: return cudaLaunchKernelEx(lc, k_spec16<float, 3, SPEC_PLAIN_INV, 7>, P, W, lgW, lax, F);
            case SPEC_GRAD: return cudaLaunchKernelEx(lc, k_spec16<float, 3, SPEC_GRAD, 7>, P, W, lgW, lax, F);
            case SPEC_DIV: return cudaLaunchKernelEx(lc, k_spec16<float, 3, SPEC_DIV, 7>, P, W, lgW, lax, F);
            case SPEC_ABS: return cudaLaunchKernelEx(lc, k_spec16<float, 3, SPEC_ABS, 7>, P, W, lgW, lax, F);
            case SPEC_DIVT: return cudaLaunchKernelEx(lc, k_spec16<float, 3, SPEC_DIVT, 7>, P, W, lgW, lax, F);
            case SPEC_GRADT: return cudaLaunchKernelEx(lc, k_spec16<float, 3, SPEC_GRADT, 7>, P, W, lgW, lax, F);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (mode) {
        case SPEC_PLAIN_FWD: return cudaLaunchKernelEx(lc, k_spec2<float, 3, SPEC_PLAIN_FWD, 7>, P, W, lgW, lax, F);
        case SPEC_PLAIN_INV: return cudaLaunchKernelEx(lc, k_spec2<float, 3, SPEC_PLAIN_INV, 7>, P, W, lgW, lax, F);
        case SPEC_GRAD: return cudaLaunchKernelEx(lc, k_spec2<float, 3, SPEC_GRAD, 7>, P, W, lgW, lax, F);
        case SPEC_DIV: return cudaLaunchKernelEx(lc, k_spec2<float, 3, SPEC_DIV, 7>, P, W, lgW, lax, F);
        case SPEC_ABS: return cudaLaunchKernelEx(lc, k_spec2<float, 3, SPEC_ABS, 7>, P, W, lgW, lax, F);
        case SPEC_DIVT: return cudaLaunchKernelEx(lc, k_spec2<float, 3, SPEC_DIVT, 7>, P, W, lgW, lax, F);
        case SPEC_GRADT: return cudaLaunchKernelEx(lc, k_spec2<float, 3, SPEC_GRADT, 7>, P, W, lgW, lax, F);
        default: return cudaErrorInvalidValue;
    }
}

template <> cudaError_t spec2_set_attrs_f32_3d<7>(int bytes) {
    const void* ks[] = {
        (const void*)k_spec2<float, 3, SPEC_PLAIN_FWD, 7>,
        (const void*)k_spec16<float, 3, SPEC_PLAIN_FWD, 7>,
        (const void*)k_spec2<float, 3, SPEC_PLAIN_INV, 7>,
        (const void*)k_spec16<float, 3, SPEC_PLAIN_INV, 7>,
        (const void*)k_spec2<float, 3, SPEC_GRAD, 7>,
        (const void*)k_spec16<float, 3, SPEC_GRAD, 7>,
        (const void*)k_spec2<float, 3, SPEC_DIV, 7>,
        (const void*)k_spec16<float, 3, SPEC_DIV, 7>,
        (const void*)k_spec2<float, 3, SPEC_ABS, 7>,
        (const void*)k_spec16<float, 3, SPEC_ABS, 7>,
        (const void*)k_spec2<float, 3, SPEC_DIVT, 7>,
        (const void*)k_spec16<float, 3, SPEC_DIVT, 7>,
        (const void*)k_spec2<float, 3, SPEC_GRADT, 7>,
        (const void*)k_spec16<float, 3, SPEC_GRADT, 7>,
    };
    for (const void* k : ks) {
        cudaError_t e = set_dyn_smem(k, bytes);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace pat
