// pat_p2.h -- host-side view of the power-of-two persistent kernel (pat_persist2.cuh): its
// shared-memory layout and its launch entry, compiled in a translation unit per precision.
#pragma once

#include <complex>
#include <type_traits>
#include <vector>

#include "pat_kernels.cuh"

namespace pat {

struct PersistCfg;

// ---- fixed power-of-two Stockham schedule ----
// nst = ceil(lg / 3) stages (lg >= 4); forward stage s: radix r0 (s = 0) or 8, Ns = 1 (s = 0) or
// r0 8^(s - 1); inverse stage s: radix 8 (s < nst - 1) or r0, Ns = 8^s.
struct P2Axis {
    int n, lg, nst, r0;
};
__host__ __device__ __forceinline__ P2Axis p2_axis(int lg) {
    P2Axis a;
    a.lg = lg;
    a.n = 1 << lg;
    a.nst = (lg + 2) / 3;
    a.r0 = 1 << (lg - 3 * (a.nst - 1));
    return a;
}
// The same schedule with the line length fixed when the kernel is compiled: every span, stride and
// table offset of a stage is then a constant, and the swizzled addresses of a butterfly are one
// per-thread base plus constant offsets.  Kernels take either type as their axis.
template <int LG> struct P2AxisC {
    static constexpr int lg = LG, n = 1 << LG, nst = (LG + 2) / 3, r0 = 1 << (LG - 3 * ((LG + 2) / 3 - 1));
};
template <class AX> struct P2IsC : std::false_type {};
template <int LG> struct P2IsC<P2AxisC<LG>> : std::true_type {};
// axis of a kernel compiled for line length 2^LG (LG = 0: any length, from the plan)
template <int LG> struct P2Sel {
    using type = P2AxisC<LG>;
    static __host__ __device__ __forceinline__ type make(int) { return type{}; }
};
template <> struct P2Sel<0> {
    using type = P2Axis;
    static __host__ __device__ __forceinline__ type make(int lg) { return p2_axis(lg); }
};

template <class AX> __host__ __device__ __forceinline__ int p2_fns(const AX& a, int s) {
    return s == 0 ? 1 : a.r0 << (3 * (s - 1));
}
__host__ __device__ __forceinline__ int p2_ins(int s) { return 1 << (3 * s); }
template <class AX> __host__ __device__ __forceinline__ int p2_ir(const AX& a, int s) {
    return s == a.nst - 1 ? a.r0 : 8;
}
// twiddle tables of one axis: forward stages 1..nst-1, then inverse stages 1..nst-1 (< 2 n entries)
template <class AX> __host__ __device__ __forceinline__ int p2_off_f(const AX& a, int s) { return p2_fns(a, s) - a.r0; }
template <class AX> __host__ __device__ __forceinline__ int p2_off_i(const AX& a, int s) {
    return a.n - a.r0 + p2_ins(s) - 8;
}

__host__ __device__ __forceinline__ int p2_tab_len(int n) { return 2 * n; }

// Stage twiddle tables of a power-of-two axis (n = 2^lg, lg >= 4) from its full table
// tw[m] = exp(-2 pi i m / n): entry (r, k) of a stage of radix R and span Ns is tw[r k n / (Ns R)].
// A gather of the same values, so the rounded tables the kernels use are those of the full table.
inline std::vector<std::complex<double>> p2_stage_table(const std::vector<std::complex<double>>& tw, int lg) {
    const P2Axis a = p2_axis(lg);
    std::vector<std::complex<double>> t((size_t)p2_tab_len(a.n), std::complex<double>(0.0, 0.0));
    for (int s = 1; s < a.nst; ++s) {
        const int NsF = p2_fns(a, s), NsI = p2_ins(s), RI = p2_ir(a, s);
        const int stepF = a.n / (NsF * 8), stepI = a.n / (NsI * RI);
        for (int r = 1; r < 8; ++r)
            for (int k = 0; k < NsF; ++k) t[(size_t)p2_off_f(a, s) + (r - 1) * NsF + k] = tw[(size_t)r * k * stepF];
        for (int r = 1; r < RI; ++r)
            for (int k = 0; k < NsI; ++k) t[(size_t)p2_off_i(a, s) + (r - 1) * NsI + k] = tw[(size_t)r * k * stepI];
    }
    return t;
}

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
// raise kernel k's dynamic shared-memory limit to `bytes` less its static shared memory (the spectral
// kernels hold the mbarrier of their tensor copies there), so that the sum stays within the opt-in limit
inline cudaError_t set_dyn_smem(const void* k, int bytes) {
    cudaFuncAttributes a{};
    cudaError_t e = cudaFuncGetAttributes(&a, k);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes - (int)a.sharedSizeBytes);
}
// k_spec2's lanes step across the tile's lines: every line is followed by 16 bytes of padding
template <typename T> __host__ __device__ __forceinline__ int spec2_line_pad() { return 16 / (int)sizeof(cplx<T>); }
// fields a k_spec2 launch holds at once: max(fields in, fields out)
__host__ __device__ __forceinline__ int spec2_nf(int D, int mode, int F) {
    if (mode == SPEC_PLAIN_FWD || mode == SPEC_PLAIN_INV) return F > 1 ? F : 1;
    return mode == SPEC_ABS ? 2 : D;
}
// shared memory of k_spec2: stage twiddle tables [2 L] | the line axis' k [L] (real) and shift
// operator [L] (complex) | A | B, each of nf W padded lines (+ 2 field pads)
template <typename T> __host__ __device__ size_t spec2_buf_elems(int nf, int L, int W) {
    return (size_t)nf * W * (L + spec2_line_pad<T>()) + 2 * (size_t)p2_field_pad<T>();
}
template <typename T> __host__ __device__ size_t spec2_pre_elems(int L) {
    return (size_t)p2_tab_len(L) + (size_t)L + ((size_t)L * sizeof(T) + sizeof(cplx<T>) - 1) / sizeof(cplx<T>);
}
template <typename T> size_t spec2_smem_bytes(int nf, int L, int W) {
    return (spec2_pre_elems<T>(L) + 2 * spec2_buf_elems<T>(nf, L, W)) * sizeof(cplx<T>);
}

// register-resident z passes of 256-point lines, float (pat_zreg.cuh): launch k_zreg<mode> with the
// grid, stream and attributes of `lc` (block size and shared memory are set here)
cudaError_t zreg_launch(const cudaLaunchConfig_t* lc, int mode, const DevPlan<float>& P);
cudaError_t zreg_set_attrs();
// plain y transforms of 128- and 256-point y-lines on 16-column tiles, float (pat_ywide.cuh): launch
// k_ywide with the grid (ceil(nxh / 16), nz, fields), stream and attributes of `lc`
cudaError_t ywide_launch(const cudaLaunchConfig_t* lc, bool inverse, const DevPlan<float>& P);
cudaError_t ywide_set_attrs();
// z passes with the k-space multiply of 128- and 256-point z-lines on 16-column tiles, float
// (pat_zwide.cuh): launch k_zwide<mode> with the grid ((fields or 1), ceil(nxh / 16), ny), stream and
// attributes of `lc`; mt = the plan's kappa / N table (zwide_kap_table, [ky][kz][ldh]) for every mode
// but SPEC_ABS, the absorption tables (zwide_abs_table, [2][ky][kz][ldh]) or nullptr for SPEC_ABS
cudaError_t zwide_launch(const cudaLaunchConfig_t* lc, int mode, const DevPlan<float>& P, const float* mt);
cudaError_t zwide_set_attrs();
cudaError_t zwide_kap_table(const DevPlan<float>& P, float* kap, cudaStream_t s);
cudaError_t zwide_abs_table(const DevPlan<float>& P, float* tab, cudaStream_t s);
// the momentum row kernels with one velocity component per CTA (pat_rowu1.cuh), float, 3-D x-lines of
// 128 and 256 points: launch k_row_u1 with the grid (nlines / R, 3), stream and attributes of `lc`
cudaError_t rowu1_launch(const cudaLaunchConfig_t* lc, bool adjoint, const DevPlan<float>& P, int R, int flag);
cudaError_t rowu1_set_attrs(int bytes);

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

// launch k_persist2<T, adjoint> with `lc` (cooperative attributes set by the caller); p2_kernel is
// the kernel that p2_launch runs for a grid of 2^lgx x 2^lgy points and P.fixed_len = fixed_len
template <typename T>
cudaError_t p2_launch(bool adjoint, const cudaLaunchConfig_t* lc, const DevPlan<T>& P, const PersistCfg& C,
                      unsigned* gbar);
template <typename T> const void* p2_kernel(bool adjoint, int lgx, int lgy, int fixed_len);

// Stage tables of the two-stage schedule of an n = R1 x 16 point axis (n = 128 or 256; forward
// radices R1, 16; inverse 16, R1): the forward radix-16 stage (span R1) [15][R1] at 0, then the
// inverse radix-R1 stage (span 16) [R1 - 1][16]; entry (r, k) is tw[r k] in both (a gather).
inline std::vector<std::complex<double>> p2x_stage_table(const std::vector<std::complex<double>>& tw, int lg) {
    const int n = 1 << lg, R1 = n / 16;
    std::vector<std::complex<double>> t((size_t)p2_tab_len(n), std::complex<double>(0.0, 0.0));
    for (int r = 1; r < 16; ++r)
        for (int k = 0; k < R1; ++k) t[(size_t)(r - 1) * R1 + k] = tw[(size_t)r * k];
    for (int r = 1; r < R1; ++r)
        for (int k = 0; k < 16; ++k) t[(size_t)15 * R1 + (r - 1) * 16 + k] = tw[(size_t)r * k];
    return t;
}

// ---- kernels compiled for fixed lengths (float fields) ----
// The 2-D persistent kernel for 256^2 and 512^2 grids, and the 3-D spectral and row kernels for
// lines of 64, 128 and 256 points; a plan takes them unless it was created with PAT_P2SPEC=0
// (DevPlan::fixed_len = 0), which runs the kernels for any length instead (for comparison).
// lg of the fixed-size 2-D persistent kernel for a 2^lgx x 2^lgy grid, 0 if there is none
inline int p2_sq_lg(int lgx, int lgy, int on) { return (on && lgx == lgy && (lgx == 8 || lgx == 9)) ? lgx : 0; }
// lg of the fixed-length 3-D spectral or row kernel for lines of 2^lg points, 0 if there is none
inline int p2_3d_lg(int lg, int on) { return (on && lg >= 6 && lg <= 8) ? lg : 0; }
template <int LG>
cudaError_t p2_launch_f32_sq(bool adjoint, const cudaLaunchConfig_t* lc, const DevPlan<float>& P, const PersistCfg& C,
                             unsigned* gbar);
template <int LG> const void* p2_kernel_f32_sq(bool adjoint);
template <int LG>
cudaError_t spec2_launch_f32_3d(const cudaLaunchConfig_t* lc, int mode, const DevPlan<float>& P, int W, int lgW, int lax,
                                int F);
template <int LG> cudaError_t spec2_set_attrs_f32_3d(int bytes);
template <int LG>
cudaError_t row2_launch_f32_3d(const cudaLaunchConfig_t* lc, int kind, const DevPlan<float>& P, int R, int flag,
                               float* data_row, const float* h_row, float* qrow, float* gc2, const float* p0c);
template <int LG> cudaError_t row2_set_attrs_f32_3d(int bytes);

}  // namespace pat
