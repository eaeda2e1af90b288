// pat_zwide_f32.cu -- the 16-column z passes of 128- and 256-point z-lines (pat_zwide.cuh), float
// fields, and their multiplier tables.
#include "pat_zwide.cuh"

namespace pat {

template <int MODE> static cudaError_t zwide_go(cudaLaunchConfig_t* lc, const DevPlan<float>& P, const float* mt) {
    lc->dynamicSmemBytes = zwide_smem_bytes<MODE>(P.nz);
    return P.nz == 256 ? cudaLaunchKernelEx(lc, k_zwide<8, MODE>, P, mt) : cudaLaunchKernelEx(lc, k_zwide<7, MODE>, P, mt);
}

cudaError_t zwide_launch(const cudaLaunchConfig_t* lc0, int mode, const DevPlan<float>& P, const float* mt) {
    cudaLaunchConfig_t lc = *lc0;
    lc.blockDim = dim3(256);
    if (P.nz != 128 && P.nz != 256) return cudaErrorInvalidValue;
    switch (mode) {
        case SPEC_GRAD: return zwide_go<SPEC_GRAD>(&lc, P, mt);
        case SPEC_DIV: return zwide_go<SPEC_DIV>(&lc, P, mt);
        case SPEC_ABS: return zwide_go<SPEC_ABS>(&lc, P, mt);
        case SPEC_DIVT: return zwide_go<SPEC_DIVT>(&lc, P, mt);
        case SPEC_GRADT: return zwide_go<SPEC_GRADT>(&lc, P, mt);
        default: return cudaErrorInvalidValue;
    }
}

template <int MODE> static cudaError_t zwide_attr() {
    cudaError_t e = cudaFuncSetAttribute(k_zwide<8, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)zwide_smem_bytes<MODE>(256));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_zwide<7, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)zwide_smem_bytes<MODE>(128));
}

cudaError_t zwide_set_attrs() {
    cudaError_t e = zwide_attr<SPEC_GRAD>();
    if (e == cudaSuccess) e = zwide_attr<SPEC_DIV>();
    if (e == cudaSuccess) e = zwide_attr<SPEC_ABS>();
    if (e == cudaSuccess) e = zwide_attr<SPEC_DIVT>();
    if (e == cudaSuccess) e = zwide_attr<SPEC_GRADT>();
    return e;
}

cudaError_t zwide_kap_table(const DevPlan<float>& P, float* kap, cudaStream_t s) {
    k_kap_table<<<4 * 152, 256, 0, s>>>(P, kap);
    return cudaGetLastError();
}

cudaError_t zwide_abs_table(const DevPlan<float>& P, float* tab, cudaStream_t s) {
    k_abs_table<<<4 * 152, 256, 0, s>>>(P, tab);
    return cudaGetLastError();
}

}  // namespace pat
