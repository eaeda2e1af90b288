// pat_zwide_f32.cu -- the 16-column z passes with a field-wise multiply on 128- and 256-point z-lines
// (pat_zwide.cuh), float fields, and their kappa table.
#include "pat_zwide.cuh"

namespace pat {

cudaError_t zwide_launch(const cudaLaunchConfig_t* lc0, int mode, const DevPlan<float>& P, const float* kap) {
    cudaLaunchConfig_t lc = *lc0;
    lc.blockDim = dim3(256);
    if (P.nz != 128 && P.nz != 256) return cudaErrorInvalidValue;
    const bool l8 = P.nz == 256;
    lc.dynamicSmemBytes = zwide_smem_bytes(P.nz);
    switch (mode) {
        case SPEC_DIV:
            return l8 ? cudaLaunchKernelEx(&lc, k_zwide<8, SPEC_DIV>, P, kap) : cudaLaunchKernelEx(&lc, k_zwide<7, SPEC_DIV>, P, kap);
        case SPEC_DIVT:
            return l8 ? cudaLaunchKernelEx(&lc, k_zwide<8, SPEC_DIVT>, P, kap)
                      : cudaLaunchKernelEx(&lc, k_zwide<7, SPEC_DIVT>, P, kap);
        case SPEC_ABS:
            return l8 ? cudaLaunchKernelEx(&lc, k_zwide<8, SPEC_ABS>, P, kap) : cudaLaunchKernelEx(&lc, k_zwide<7, SPEC_ABS>, P, kap);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t zwide_set_attrs() {
    struct K {
        const void* k;
        size_t bytes;
    } ks[] = {
        {(const void*)k_zwide<8, SPEC_DIV>, zwide_smem_bytes(256)},  {(const void*)k_zwide<8, SPEC_DIVT>, zwide_smem_bytes(256)},
        {(const void*)k_zwide<8, SPEC_ABS>, zwide_smem_bytes(256)},  {(const void*)k_zwide<7, SPEC_DIV>, zwide_smem_bytes(128)},
        {(const void*)k_zwide<7, SPEC_DIVT>, zwide_smem_bytes(128)}, {(const void*)k_zwide<7, SPEC_ABS>, zwide_smem_bytes(128)},
    };
    for (const K& k : ks) {
        cudaError_t e = cudaFuncSetAttribute(k.k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.bytes);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t zwide_kap_table(const DevPlan<float>& P, float* kap, cudaStream_t s) {
    k_kap_table<<<4 * 152, 256, 0, s>>>(P, kap);
    return cudaGetLastError();
}

}  // namespace pat
