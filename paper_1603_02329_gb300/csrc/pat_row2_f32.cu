// pat_row2_f32.cu -- the power-of-two row kernels instantiated for float fields.
#include "pat_row2.cuh"

namespace pat {

template <>
cudaError_t row2_launch<float>(const cudaLaunchConfig_t* lc, int D, int kind, const DevPlan<float>& P, int R, int flag,
                            float* data_row, const float* h_row, float* qrow, float* gc2, const float* p0c) {
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
    return cudaSuccess;
}

}  // namespace pat
