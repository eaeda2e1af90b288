// pat_row2_f32_n64.cu -- the 3-D power-of-two row kernels compiled for x-lines of 64 points, float
// fields.
#include "pat_row2.cuh"

namespace pat {

template <>
cudaError_t row2_launch_f32_3d<6>(const cudaLaunchConfig_t* lc, int kind, const DevPlan<float>& P, int R, int flag,
                                   float* data_row, const float* h_row, float* qrow, float* gc2, const float* p0c) {
    switch (kind) {
        case R2_FWD_U:
            return cudaLaunchKernelEx(lc, k_row2<float, 3, R2_FWD_U, 6>, P, R, flag, data_row, h_row, qrow, gc2, p0c);
        case R2_FWD_RHO:
            return cudaLaunchKernelEx(lc, k_row2<float, 3, R2_FWD_RHO, 6>, P, R, flag, data_row, h_row, qrow, gc2, p0c);
        case R2_FWD_P:
            return cudaLaunchKernelEx(lc, k_row2<float, 3, R2_FWD_P, 6>, P, R, flag, data_row, h_row, qrow, gc2, p0c);
        case R2_ADJ_RHO:
            return cudaLaunchKernelEx(lc, k_row2<float, 3, R2_ADJ_RHO, 6>, P, R, flag, data_row, h_row, qrow, gc2, p0c);
        case R2_ADJ_U:
            return cudaLaunchKernelEx(lc, k_row2<float, 3, R2_ADJ_U, 6>, P, R, flag, data_row, h_row, qrow, gc2, p0c);
        case R2_ADJ_P:
            return cudaLaunchKernelEx(lc, k_row2<float, 3, R2_ADJ_P, 6>, P, R, flag, data_row, h_row, qrow, gc2, p0c);
        default: return cudaErrorInvalidValue;
    }
}

template <> cudaError_t row2_set_attrs_f32_3d<6>(int bytes) {
    const void* ks[] = {
        (const void*)k_row2<float, 3, R2_FWD_U, 6>,
        (const void*)k_row2<float, 3, R2_FWD_RHO, 6>,
        (const void*)k_row2<float, 3, R2_FWD_P, 6>,
        (const void*)k_row2<float, 3, R2_ADJ_RHO, 6>,
        (const void*)k_row2<float, 3, R2_ADJ_U, 6>,
        (const void*)k_row2<float, 3, R2_ADJ_P, 6>,
    };
    for (const void* k : ks) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace pat
