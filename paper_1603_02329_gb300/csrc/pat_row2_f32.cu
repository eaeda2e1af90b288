// pat_row2_f32.cu -- the power-of-two row kernels instantiated for float fields (any length; 3-D
// x-lines of 64, 128 and 256 points run the fixed-length instances of pat_row2_f32_n*.cu).
#include "pat_row2.cuh"

namespace pat {

template <>
cudaError_t row2_launch<float>(const cudaLaunchConfig_t* lc, int D, int kind, const DevPlan<float>& P, int R, int flag,
                            float* data_row, const float* h_row, float* qrow, float* gc2, const float* p0c) {
    if (D == 3) {
        switch (p2_3d_lg(P.fx.lgn, P.fixed_len)) {
            case 6: return row2_launch_f32_3d<6>(lc, kind, P, R, flag, data_row, h_row, qrow, gc2, p0c);
            case 7: return row2_launch_f32_3d<7>(lc, kind, P, R, flag, data_row, h_row, qrow, gc2, p0c);
            case 8: return row2_launch_f32_3d<8>(lc, kind, P, R, flag, data_row, h_row, qrow, gc2, p0c);
            default: break;
        }
    }
    switch (D * 8 + kind) {
        case 2 * 8 + R2_FWD_U:
            return cudaLaunchKernelEx(lc, k_row2<float, 2, R2_FWD_U>, P, R, flag, data_row, h_row, qrow, gc2, p0c);
        case 2 * 8 + R2_FWD_RHO:
            return cudaLaunchKernelEx(lc, k_row2<float, 2, R2_FWD_RHO>, P, R, flag, data_row, h_row, qrow, gc2, p0c);
        case 2 * 8 + R2_FWD_P:
            return cudaLaunchKernelEx(lc, k_row2<float, 2, R2_FWD_P>, P, R, flag, data_row, h_row, qrow, gc2, p0c);
        case 2 * 8 + R2_ADJ_RHO:
            return cudaLaunchKernelEx(lc, k_row2<float, 2, R2_ADJ_RHO>, P, R, flag, data_row, h_row, qrow, gc2, p0c);
        case 2 * 8 + R2_ADJ_U:
            return cudaLaunchKernelEx(lc, k_row2<float, 2, R2_ADJ_U>, P, R, flag, data_row, h_row, qrow, gc2, p0c);
        case 2 * 8 + R2_ADJ_P:
            return cudaLaunchKernelEx(lc, k_row2<float, 2, R2_ADJ_P>, P, R, flag, data_row, h_row, qrow, gc2, p0c);
        case 3 * 8 + R2_FWD_U:
            return cudaLaunchKernelEx(lc, k_row2<float, 3, R2_FWD_U>, P, R, flag, data_row, h_row, qrow, gc2, p0c);
        case 3 * 8 + R2_FWD_RHO:
            return cudaLaunchKernelEx(lc, k_row2<float, 3, R2_FWD_RHO>, P, R, flag, data_row, h_row, qrow, gc2, p0c);
        case 3 * 8 + R2_FWD_P:
            return cudaLaunchKernelEx(lc, k_row2<float, 3, R2_FWD_P>, P, R, flag, data_row, h_row, qrow, gc2, p0c);
        case 3 * 8 + R2_ADJ_RHO:
            return cudaLaunchKernelEx(lc, k_row2<float, 3, R2_ADJ_RHO>, P, R, flag, data_row, h_row, qrow, gc2, p0c);
        case 3 * 8 + R2_ADJ_U:
            return cudaLaunchKernelEx(lc, k_row2<float, 3, R2_ADJ_U>, P, R, flag, data_row, h_row, qrow, gc2, p0c);
        case 3 * 8 + R2_ADJ_P:
            return cudaLaunchKernelEx(lc, k_row2<float, 3, R2_ADJ_P>, P, R, flag, data_row, h_row, qrow, gc2, p0c);
        default: return cudaErrorInvalidValue;
    }
}

template <> cudaError_t row2_set_attrs<float>(int bytes) {
    const void* ks[] = {
        (const void*)k_row2<float, 2, R2_FWD_U>,
        (const void*)k_row2<float, 2, R2_FWD_RHO>,
        (const void*)k_row2<float, 2, R2_FWD_P>,
        (const void*)k_row2<float, 2, R2_ADJ_RHO>,
        (const void*)k_row2<float, 2, R2_ADJ_U>,
        (const void*)k_row2<float, 2, R2_ADJ_P>,
        (const void*)k_row2<float, 3, R2_FWD_U>,
        (const void*)k_row2<float, 3, R2_FWD_RHO>,
        (const void*)k_row2<float, 3, R2_FWD_P>,
        (const void*)k_row2<float, 3, R2_ADJ_RHO>,
        (const void*)k_row2<float, 3, R2_ADJ_U>,
        (const void*)k_row2<float, 3, R2_ADJ_P>,
    };
    for (const void* k : ks) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = row2_set_attrs_f32_3d<6>(bytes);
    if (e == cudaSuccess) e = row2_set_attrs_f32_3d<7>(bytes);
    if (e == cudaSuccess) e = row2_set_attrs_f32_3d<8>(bytes);
    return e;
}

}  // namespace pat
