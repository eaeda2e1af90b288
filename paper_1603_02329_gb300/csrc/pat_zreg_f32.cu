// pat_zreg_f32.cu -- the register-resident z passes of 256-point lines (pat_zreg.cuh), float fields.
#include "pat_zreg.cuh"

namespace pat {

cudaError_t zreg_launch(const cudaLaunchConfig_t* lc0, int mode, const DevPlan<float>& P) {
    cudaLaunchConfig_t lc = *lc0;
    switch (mode) {
        case SPEC_GRAD:
            lc.blockDim = dim3(128 * ZregDims<SPEC_GRAD>::NF);
            lc.dynamicSmemBytes = zreg_smem_bytes<SPEC_GRAD>();
            return cudaLaunchKernelEx(&lc, k_zreg<SPEC_GRAD>, P);
        case SPEC_DIV:
            lc.blockDim = dim3(128 * ZregDims<SPEC_DIV>::NF);
            lc.dynamicSmemBytes = zreg_smem_bytes<SPEC_DIV>();
            return cudaLaunchKernelEx(&lc, k_zreg<SPEC_DIV>, P);
        case SPEC_ABS:
            lc.blockDim = dim3(128 * ZregDims<SPEC_ABS>::NF);
            lc.dynamicSmemBytes = zreg_smem_bytes<SPEC_ABS>();
            return cudaLaunchKernelEx(&lc, k_zreg<SPEC_ABS>, P);
        case SPEC_DIVT:
            lc.blockDim = dim3(128 * ZregDims<SPEC_DIVT>::NF);
            lc.dynamicSmemBytes = zreg_smem_bytes<SPEC_DIVT>();
            return cudaLaunchKernelEx(&lc, k_zreg<SPEC_DIVT>, P);
        case SPEC_GRADT:
            lc.blockDim = dim3(128 * ZregDims<SPEC_GRADT>::NF);
            lc.dynamicSmemBytes = zreg_smem_bytes<SPEC_GRADT>();
            return cudaLaunchKernelEx(&lc, k_zreg<SPEC_GRADT>, P);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t zreg_set_attrs() {
    struct K {
        const void* k;
        size_t bytes;
    } ks[] = {
        {(const void*)k_zreg<SPEC_GRAD>, zreg_smem_bytes<SPEC_GRAD>()},
        {(const void*)k_zreg<SPEC_DIV>, zreg_smem_bytes<SPEC_DIV>()},
        {(const void*)k_zreg<SPEC_ABS>, zreg_smem_bytes<SPEC_ABS>()},
        {(const void*)k_zreg<SPEC_DIVT>, zreg_smem_bytes<SPEC_DIVT>()},
        {(const void*)k_zreg<SPEC_GRADT>, zreg_smem_bytes<SPEC_GRADT>()},
    };
    for (const K& k : ks) {
        cudaError_t e = cudaFuncSetAttribute(k.k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.bytes);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace pat
