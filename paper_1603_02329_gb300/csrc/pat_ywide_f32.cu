// pat_ywide_f32.cu -- the 16-column plain y transforms of 128- and 256-point y-lines (pat_ywide.cuh),
// float fields.
#include "pat_ywide.cuh"

namespace pat {

cudaError_t ywide_launch(const cudaLaunchConfig_t* lc0, bool inverse, const DevPlan<float>& P) {
    cudaLaunchConfig_t lc = *lc0;
    lc.blockDim = dim3(256);
    if (P.ny == 256) {
        lc.dynamicSmemBytes = ywide_smem_bytes(256);
        return inverse ? cudaLaunchKernelEx(&lc, k_ywide<8, true>, P) : cudaLaunchKernelEx(&lc, k_ywide<8, false>, P);
    }
    if (P.ny == 128) {
        lc.dynamicSmemBytes = ywide_smem_bytes(128);
        return inverse ? cudaLaunchKernelEx(&lc, k_ywide<7, true>, P) : cudaLaunchKernelEx(&lc, k_ywide<7, false>, P);
    }
    return cudaErrorInvalidValue;
}

cudaError_t ywide_set_attrs() {
    struct K {
        const void* k;
        size_t bytes;
    } ks[] = {
        {(const void*)k_ywide<8, false>, ywide_smem_bytes(256)},
        {(const void*)k_ywide<8, true>, ywide_smem_bytes(256)},
        {(const void*)k_ywide<7, false>, ywide_smem_bytes(128)},
        {(const void*)k_ywide<7, true>, ywide_smem_bytes(128)},
    };
    for (const K& k : ks) {
        cudaError_t e = cudaFuncSetAttribute(k.k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.bytes);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace pat
