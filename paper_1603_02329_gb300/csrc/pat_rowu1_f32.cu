// pat_rowu1_f32.cu -- the one-component momentum row kernels (pat_rowu1.cuh) for float fields and
// 3-D x-lines of 128 and 256 points.
#include "pat_rowu1.cuh"

namespace pat {

cudaError_t rowu1_launch(const cudaLaunchConfig_t* lc0, bool adjoint, const DevPlan<float>& P, int R, int flag) {
    cudaLaunchConfig_t lc = *lc0;
    lc.blockDim = dim3(256);
    lc.dynamicSmemBytes = rowu1_layout<float>(P.nx, P.ldh, R).bytes;
    switch (P.fx.lgn * 2 + (adjoint ? 1 : 0)) {
        case 14: return cudaLaunchKernelEx(&lc, k_row_u1<float, 7, false>, P, R, flag);
        case 15: return cudaLaunchKernelEx(&lc, k_row_u1<float, 7, true>, P, R, flag);
        case 16: return cudaLaunchKernelEx(&lc, k_row_u1<float, 8, false>, P, R, flag);
        case 17: return cudaLaunchKernelEx(&lc, k_row_u1<float, 8, true>, P, R, flag);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t rowu1_set_attrs(int bytes) {
    const void* ks[] = {(const void*)k_row_u1<float, 7, false>, (const void*)k_row_u1<float, 7, true>,
                        (const void*)k_row_u1<float, 8, false>, (const void*)k_row_u1<float, 8, true>};
    for (const void* k : ks) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace pat
