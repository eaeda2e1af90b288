// pat_smooth.cu -- the optional smoothing S of the initial pressure (Sec. VI.A: the high
// frequencies of p0 are filtered by a self-adjoint operator before every forward solve, and the
// same operator closes the adjoint).
//
// S = F^-1 diag(W) F with the radial Blackman window W(k) = B(|k| / k_c),
// B(q) = 0.42 + 0.5 cos(pi q) + 0.08 cos(2 pi q) for q < 1 and 0 beyond, k_c the smallest per-axis
// Nyquist wavenumber pi / dx.  W is real, even in k and in [0, 1]: S is real, symmetric and
// non-expansive, so the smoothed operator is H S and its transpose S H^T.
//
// S runs once per solve (against Nt time steps), so it favours plainness over speed: full
// complex transforms of the real field, one axis per launch, through the library's Stockham
// routines (pat_fft.cuh) and the plan's FFT plans and twiddles.  Passes, for a field x (in place):
//   rows   x-lines of x -> forward transform -> workspace Z        (complex [nz][ny][nx])
//   cols   y (2-D: forward, window, inverse; 3-D: forward) on Z
//   cols   z forward, window, inverse on Z                         (3-D only)
//   cols   y inverse on Z                                          (3-D only)
//   rows   x-lines of Z -> inverse transform -> real part into x
// The window multiply carries the 1 / N of the unnormalised inverse transforms.  Shared memory
// stays within the 48 KB that needs no opt-in; every access is guarded by the line / column count.
#include <algorithm>

#include "pat_fft.cuh"
#include "pat_smooth.h"

namespace pat {

namespace {

constexpr int kSmThreads = 256;
constexpr size_t kSmSmem = 48 * 1024;

// signed wavenumber index of bin m on an axis of n points (Nyquist bin positive)
__device__ __forceinline__ int signed_bin(int m, int n) { return (m <= n / 2) ? m : m - n; }

// W(k) / N at bins (mx, my, mz), in FP64
template <typename T> __device__ __forceinline__ double window_over_n(const SmoothArgs<T>& A, int mx, int my, int mz) {
    const double kx = signed_bin(mx, A.nx) * A.dk[0];
    const double ky = signed_bin(my, A.ny) * A.dk[1];
    const double kz = (A.d == 3) ? signed_bin(mz, A.nz) * A.dk[2] : 0.0;
    const double q2 = (kx * kx + ky * ky + kz * kz) * A.inv_kc2;
    if (q2 >= 1.0) return 0.0;
    const double q = sqrt(q2);
    return (0.42 + 0.5 * cospi(q) + 0.08 * cospi(2.0 * q)) * A.invN;
}

// x-lines [line0, line0 + cnt) of the field: forward (x real -> Z) or inverse (Z -> real part of x)
template <typename T, bool INV>
__global__ void __launch_bounds__(kSmThreads) k_sm_rows(SmoothArgs<T> A, T* x, int nl) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nx = A.nx;
    cplx<T>* a = reinterpret_cast<cplx<T>*>(smem_raw);
    cplx<T>* b = a + (size_t)nl * nx;
    const int nlines = A.ny * A.nz;
    const int line0 = blockIdx.x * nl;
    if (line0 >= nlines) return;
    const int cnt = min(nl, nlines - line0);
    const size_t off = (size_t)line0 * nx;
    for (int t = threadIdx.x; t < cnt * nx; t += blockDim.x)
        a[t] = INV ? A.Z[off + t] : mkc<T>(x[off + t], (T)0);
    __syncthreads();
    const cplx<T>* r = fft_rows<T, INV>(a, b, A.ax[0], A.tw[0], cnt);
    for (int t = threadIdx.x; t < cnt * nx; t += blockDim.x) {
        if (INV) x[off + t] = r[t].x;
        else A.Z[off + t] = r[t];
    }
}

// Lines of Z along axis lax (1: y, 2: z) through the W columns x0 .. x0 + W - 1 at outer index
// blockIdx.y (z for lax = 1, y for lax = 2).  MODE 0: forward transform; 1: inverse; 2: forward,
// window / N, inverse.
template <typename T, int MODE>
__global__ void __launch_bounds__(kSmThreads) k_sm_cols(SmoothArgs<T> A, int lax, int W, int lgW) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const FftAxis& ax = A.ax[lax];
    const int n = ax.n;
    cplx<T>* a = reinterpret_cast<cplx<T>*>(smem_raw);
    cplx<T>* b = a + (size_t)n * W;
    const int x0 = blockIdx.x * W, outer = blockIdx.y;
    if (x0 >= A.nx) return;
    const int wv = min(W, A.nx - x0);
    const size_t es = (lax == 1) ? (size_t)A.nx : (size_t)A.ny * A.nx;
    const size_t base = (lax == 1) ? (size_t)outer * A.ny * A.nx + x0 : (size_t)outer * A.nx + x0;
    // element e of column c at a[c + e W]
    for (int t = threadIdx.x; t < n * W; t += blockDim.x) {
        const int e = t >> lgW, c = t & (W - 1);
        a[t] = (c < wv) ? A.Z[base + (size_t)e * es + c] : mkc<T>((T)0, (T)0);
    }
    __syncthreads();
    cplx<T>* r = fft_cols<T, MODE == 1>(a, b, ax, A.tw[lax], W, lgW);
    if constexpr (MODE == 2) {
        for (int t = threadIdx.x; t < n * W; t += blockDim.x) {
            const int e = t >> lgW, c = t & (W - 1);
            const int mx = min(x0 + c, A.nx - 1);
            const double w = (lax == 1) ? window_over_n(A, mx, e, outer) : window_over_n(A, mx, outer, e);
            r[t] = cscale(r[t], (T)w);
        }
        __syncthreads();
        cplx<T>* other = (r == a) ? b : a;
        r = fft_cols<T, true>(r, other, ax, A.tw[lax], W, lgW);
    }
    for (int t = threadIdx.x; t < n * W; t += blockDim.x) {
        const int e = t >> lgW, c = t & (W - 1);
        if (c < wv) A.Z[base + (size_t)e * es + c] = r[t];
    }
}

// x-lines per row CTA: two complex buffers of nl lines within the shared-memory budget
int rows_per_cta(int nx, size_t elem) {
    const size_t per_line = 2 * (size_t)nx * 2 * elem;
    return (int)std::max<size_t>(1, std::min<size_t>(16, kSmSmem / per_line));
}

// columns per column CTA: the largest power of two <= 16 whose two buffers fit
int cols_per_cta(int n, size_t elem, int* lgW) {
    int W = 16, lg = 4;
    while (W > 1 && 2 * (size_t)n * W * 2 * elem > kSmSmem) {
        W >>= 1;
        --lg;
    }
    *lgW = lg;
    return W;
}

template <typename T> cudaError_t launch_cols(const SmoothArgs<T>& A, int mode, int lax, cudaStream_t s) {
    const int n = A.ax[lax].n;
    int lgW = 0;
    const int W = cols_per_cta(n, sizeof(T), &lgW);
    const dim3 grid((A.nx + W - 1) / W, lax == 1 ? A.nz : A.ny);
    const size_t smem = 2 * (size_t)n * W * sizeof(cplx<T>);
    if (mode == 0) k_sm_cols<T, 0><<<grid, kSmThreads, smem, s>>>(A, lax, W, lgW);
    else if (mode == 1) k_sm_cols<T, 1><<<grid, kSmThreads, smem, s>>>(A, lax, W, lgW);
    else k_sm_cols<T, 2><<<grid, kSmThreads, smem, s>>>(A, lax, W, lgW);
    return cudaGetLastError();
}

}  // namespace

template <typename T> cudaError_t smooth_apply(const SmoothArgs<T>& A, T* x, cudaStream_t s) {
    const int nl = rows_per_cta(A.nx, sizeof(T));
    const int nlines = A.ny * A.nz;
    const dim3 rgrid((nlines + nl - 1) / nl);
    const size_t rsmem = 2 * (size_t)nl * A.nx * sizeof(cplx<T>);
    k_sm_rows<T, false><<<rgrid, kSmThreads, rsmem, s>>>(A, x, nl);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (A.d == 2) {
        e = launch_cols(A, 2, 1, s);
    } else {
        e = launch_cols(A, 0, 1, s);
        if (e == cudaSuccess) e = launch_cols(A, 2, 2, s);
        if (e == cudaSuccess) e = launch_cols(A, 1, 1, s);
    }
    if (e != cudaSuccess) return e;
    k_sm_rows<T, true><<<rgrid, kSmThreads, rsmem, s>>>(A, x, nl);
    return cudaGetLastError();
}

template cudaError_t smooth_apply<float>(const SmoothArgs<float>&, float*, cudaStream_t);
template cudaError_t smooth_apply<double>(const SmoothArgs<double>&, double*, cudaStream_t);

}  // namespace pat
