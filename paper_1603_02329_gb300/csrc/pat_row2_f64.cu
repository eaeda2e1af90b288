// pat_row2_f64.cu -- the power-of-two row kernels instantiated for double fields.
#include "pat_row2.cuh"

namespace pat {

template <>
cudaError_t row2_launch<double>(const cudaLaunchConfig_t* lc, int D, int kind, const DevPlan<double>& P, int R, int flag,
                            double* data_row, const double* h_row, double* qrow, double* gc2, const double* p0c) {
    switch (D * 8 + kind) {
        case 2 * 8 + R2_FWD_U:
            return cudaLaunchKernelEx(lc, k_row2<double, 2, R2_FWD_U>, P, R, flag, data_row, h_row, qrow, gc2, p0c);
        case 2 * 8 + R2_FWD_RHO:
            return cudaLaunchKernelEx(lc, k_row2<double, 2, R2_FWD_RHO>, P, R, flag, data_row, h_row, qrow, gc2, p0c);
        case 2 * 8 + R2_FWD_P:
            return cudaLaunchKernelEx(lc, k_row2<double, 2, R2_FWD_P>, P, R, flag, data_row, h_row, qrow, gc2, p0c);
        case 2 * 8 + R2_ADJ_RHO:
            return cudaLaunchKernelEx(lc, k_row2<double, 2, R2_ADJ_RHO>, P, R, flag, data_row, h_row, qrow, gc2, p0c);
        case 2 * 8 + R2_ADJ_U:
            return cudaLaunchKernelEx(lc, k_row2<double, 2, R2_ADJ_U>, P, R, flag, data_row, h_row, qrow, gc2, p0c);
        case 2 * 8 + R2_ADJ_P:
            return cudaLaunchKernelEx(lc, k_row2<double, 2, R2_ADJ_P>, P, R, flag, data_row, h_row, qrow, gc2, p0c);
        case 3 * 8 + R2_FWD_U:
            return cudaLaunchKernelEx(lc, k_row2<double, 3, R2_FWD_U>, P, R, flag, data_row, h_row, qrow, gc2, p0c);
        case 3 * 8 + R2_FWD_RHO:
            return cudaLaunchKernelEx(lc, k_row2<double, 3, R2_FWD_RHO>, P, R, flag, data_row, h_row, qrow, gc2, p0c);
        case 3 * 8 + R2_FWD_P:
            return cudaLaunchKernelEx(lc, k_row2<double, 3, R2_FWD_P>, P, R, flag, data_row, h_row, qrow, gc2, p0c);
        case 3 * 8 + R2_ADJ_RHO:
            return cudaLaunchKernelEx(lc, k_row2<double, 3, R2_ADJ_RHO>, P, R, flag, data_row, h_row, qrow, gc2, p0c);
        case 3 * 8 + R2_ADJ_U:
            return cudaLaunchKernelEx(lc, k_row2<double, 3, R2_ADJ_U>, P, R, flag, data_row, h_row, qrow, gc2, p0c);
        case 3 * 8 + R2_ADJ_P:
            return cudaLaunchKernelEx(lc, k_row2<double, 3, R2_ADJ_P>, P, R, flag, data_row, h_row, qrow, gc2, p0c);
        default: return cudaErrorInvalidValue;
    }
}

template <> cudaError_t row2_set_attrs<double>(int bytes) {
    const void* ks[] = {
        (const void*)k_row2<double, 2, R2_FWD_U>,
        (const void*)k_row2<double, 2, R2_FWD_RHO>,
        (const void*)k_row2<double, 2, R2_FWD_P>,
        (const void*)k_row2<double, 2, R2_ADJ_RHO>,
        (const void*)k_row2<double, 2, R2_ADJ_U>,
        (const void*)k_row2<double, 2, R2_ADJ_P>,
        (const void*)k_row2<double, 3, R2_FWD_U>,
        (const void*)k_row2<double, 3, R2_FWD_RHO>,
        (const void*)k_row2<double, 3, R2_FWD_P>,
        (const void*)k_row2<double, 3, R2_ADJ_RHO>,
        (const void*)k_row2<double, 3, R2_ADJ_U>,
        (const void*)k_row2<double, 3, R2_ADJ_P>,
    };
    for (const void* k : ks) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace pat
