// pat_p2.h -- host-side view of the power-of-two persistent kernel (pat_persist2.cuh): its
// shared-memory layout and its launch entry, compiled in a translation unit per precision.
#pragma once

#include "pat_kernels.cuh"

namespace pat {

struct PersistCfg;

__host__ __device__ __forceinline__ int p2_tab_len(int n) { return 2 * n; }

// ---- shared-memory layout (pow2 kernel) ----
// twx[2 nx] | twy[2 ny] | dpl[ny] | dml[ny] | cdp[8] | cdm[8] | work | gb[rmax / 2 nx] (complex)
// | res[nres][rmax][nx] | ax, aux[nx] | ay, auy | kl2 | ckx2 | kapt [, s0t, s1t] [ny][W] | seg_w (real)
// | seg_i | flag (int)
// 64 bytes between the fields of a line buffer, in complex elements
template <typename T> __host__ __device__ __forceinline__ int p2_field_pad() { return 64 / (int)sizeof(cplx<T>); }

// work area: row phase A[rmax nx + pad] | B, where B also receives the staged half spectra of the
// rows (2 rmax ldh >= rmax nx + pad); column phase A[2 W ny + pad] | B[2 W ny + pad], B also
// receiving the staged columns
template <typename T> __host__ __device__ size_t p2_work_elems(int nx, int ny, int ldh, int rmax, int W) {
    const size_t pad = (size_t)p2_field_pad<T>();
    const size_t rowp = (size_t)rmax * nx + pad + (size_t)2 * rmax * ldh;
    const size_t colp = (size_t)2 * (2 * (size_t)W * ny + pad);
    return rowp > colp ? rowp : colp;
}
template <typename T> size_t p2_smem_bytes(int nx, int ny, int ldh, int rmax, int W, int nres, int nmul) {
    size_t b = (size_t)(p2_tab_len(nx) + p2_tab_len(ny) + 2 * ny + 16 + p2_work_elems<T>(nx, ny, ldh, rmax, W) +
                        (size_t)(rmax / 2) * nx) *
               sizeof(cplx<T>);
    b += (size_t)((size_t)nres * rmax * nx + 2 * nx + 2 * ((rmax + 3) & ~3) + ((ny + 3) & ~3) + 8 +
                  (size_t)nmul * (((size_t)W * ny + 3) & ~(size_t)3) + 2 * kSegCap) *
         sizeof(T);
    b += (size_t)(2 * kSegCap + 4) * sizeof(int);
    return b;
}

// spectral kernel of the per-phase path for power-of-two lines (pat_spec2.cuh): launch k_spec2<T, D,
// mode> with `lc` (attributes set by the caller), and raise its dynamic shared-memory limit
template <typename T>
cudaError_t spec2_launch(const cudaLaunchConfig_t* lc, int D, int mode, const DevPlan<T>& P, int W, int lgW, int lax,
                         int F);
template <typename T> cudaError_t spec2_set_attrs(int bytes);
// k_spec2's lanes step across the tile's lines: every line is followed by 16 bytes of padding
template <typename T> __host__ __device__ __forceinline__ int spec2_line_pad() { return 16 / (int)sizeof(cplx<T>); }
// shared memory of k_spec2: stage twiddle tables [2 L] | A | B, each of fmax W padded lines (+ 2
// field pads)
template <typename T> __host__ __device__ size_t spec2_buf_elems(int D, int L, int W) {
    const int fmax = D > 2 ? D : 2;
    return (size_t)fmax * W * (L + spec2_line_pad<T>()) + 2 * (size_t)p2_field_pad<T>();
}
template <typename T> size_t spec2_smem_bytes(int D, int L, int W) {
    return ((size_t)p2_tab_len(L) + 2 * spec2_buf_elems<T>(D, L, W)) * sizeof(cplx<T>);
}

// row kernels of the per-phase path for power-of-two x-lines (pat_row2.cuh)
enum Row2Kind : int { R2_FWD_U = 0, R2_FWD_RHO, R2_FWD_P, R2_ADJ_RHO, R2_ADJ_U, R2_ADJ_P };
// shared memory of k_row2: stage twiddle tables | A | B (also the staging of the spectra) | gb
// (complex), then the staged real fields and the PML factors
template <typename T> struct Row2Layout {
    size_t tab, lines, bsz, gb, res, pml, bytes;
};
template <typename T> __host__ __device__ Row2Layout<T> row2_layout(int D, int nx, int ldh, int R) {
    Row2Layout<T> L;
    const int fmax = D > 2 ? D : 2, np = R / 2;
    L.tab = (size_t)2 * nx;
    L.lines = (size_t)fmax * np * nx + 2 * (size_t)p2_field_pad<T>();
    const size_t stg = (size_t)fmax * R * ldh;
    L.bsz = L.lines > stg ? L.lines : stg;
    L.gb = (size_t)np * nx;
    const size_t ncplx = L.tab + L.lines + L.bsz + L.gb;
    L.res = (size_t)6 * R * nx;                       // at most six staged real fields
    L.pml = (size_t)nx + (((size_t)(D - 1) * R + 3) & ~(size_t)3);
    L.bytes = ncplx * sizeof(cplx<T>) + (L.res + L.pml) * sizeof(T);
    return L;
}
template <typename T>
cudaError_t row2_launch(const cudaLaunchConfig_t* lc, int D, int kind, const DevPlan<T>& P, int R, int flag,
                        T* data_row, const T* h_row, T* qrow, T* gc2, const T* p0c);
template <typename T> cudaError_t row2_set_attrs(int bytes);

// launch k_persist2<T, adjoint> with `lc` (cooperative attributes set by the caller)
template <typename T>
cudaError_t p2_launch(bool adjoint, const cudaLaunchConfig_t* lc, const DevPlan<T>& P, const PersistCfg& C,
                      unsigned* gbar);
template <typename T> const void* p2_kernel(bool adjoint);

}  // namespace pat
