// pat_kernels.cuh -- the time-stepping kernels of the forward operator and its transpose.
//
// One time step of the k-space scheme (Sec. II.A; the discrete scheme is restated in the
// library's design notes) needs three spectral operations:
//   (1) g_xi = D+_xi p            (staggered gradient, momentum equation Eq. (mom))
//   (2) e_xi = D-_xi u_xi         (staggered divergence, mass equation Eq. (mass))
//   (3) L_{y-2} dd, L_{y-1} r     (fractional Laplacians of Eq. (state); lossy media only)
// Each spectral operation is  x-FFT -> [y-FFT -> multiply -> y-IFFT] -> x-IFFT.  The x
// transforms run in "row" kernels, where the pointwise physics of the step is fused between
// the inverse transform of one operation and the forward transform of the next, so every
// state field is read and written once per step.  The middle part runs in "spectral" kernels
// over tiles of half-spectrum columns.  Two real lines share one complex transform.
#pragma once

#include "pat_fft.cuh"

namespace pat {

enum SpecMode : int {
    SPEC_PLAIN_FWD = 0,  // forward transform of F fields along the line axis
    SPEC_PLAIN_INV = 1,  // inverse transform of F fields
    SPEC_GRAD = 2,       // 1 -> d :  out_xi = D+_xi kappa / N * in            (forward (1))
    SPEC_DIV = 3,        // d -> d :  out_xi = D-_xi kappa / N * in_xi         (forward (2))
    SPEC_ABS = 4,        // 2 -> 2 :  out_0 = |k|^(y-2)/N in_0, out_1 = |k|^(y-1)/N in_1  (3)
    SPEC_DIVT = 5,       // d -> d :  out_xi = -D+_xi kappa / N * in_xi  ((D-)^T = -D+)
    SPEC_GRADT = 6       // d -> 1 :  out = -sum_xi D-_xi kappa / N * in_xi  ((D+)^T = -D-)
};

// real value of item q (= field * rows + row) at position i: items 2p, 2p+1 share complex line p
template <typename C> __device__ __forceinline__ auto& slot(C* buf, int q, int i, int nx) {
    C& c = buf[(q >> 1) * nx + i];
    return (q & 1) ? c.y : c.x;
}

template <typename C> __device__ __forceinline__ void load_tw(C* dst, const C* src, int n) {
    for (int t = threadIdx.x; t < n; t += blockDim.x) dst[t] = src[t];
}

// Pack F half-spectrum fields (x-lines line0 .. line0+R-1) into Q = F R / 2 complex lines so that
// one inverse transform per line yields two real lines (C2R of two Hermitian half spectra).
template <typename C>
__device__ void c2r_pack(C* Z, C* const* spec, int F, int R, int line0, int nx, int ldh) {
    using T = decltype(Z->x);
    const int nxh = nx / 2 + 1, Q = F * R / 2, half = nx / 2;
    for (int t = threadIdx.x; t < Q * nxh; t += blockDim.x) {
        const int p = t / nxh, k = t - p * nxh;
        const int q0 = 2 * p, q1 = 2 * p + 1;
        C A = spec[q0 / R][(size_t)(line0 + q0 % R) * ldh + k];
        C B = spec[q1 / R][(size_t)(line0 + q1 % R) * ldh + k];
        if (k == 0 || k == half) {
            A.y = 0;
            B.y = 0;
        }
        Z[p * nx + k] = mkc<T>(A.x - B.y, A.y + B.x);                     // A + i B
        if (k > 0 && k < half) Z[p * nx + nx - k] = mkc<T>(A.x + B.y, B.x - A.y);  // conj(A) + i conj(B)
    }
}

// Split Q forward-transformed complex lines (two real lines each) into F half spectra.
template <typename C>
__device__ void r2c_unpack(const C* Z, C* const* spec, int F, int R, int line0, int nx, int ldh) {
    using T = decltype(Z->x);
    const int nxh = nx / 2 + 1, Q = F * R / 2;
    for (int t = threadIdx.x; t < Q * nxh; t += blockDim.x) {
        const int p = t / nxh, k = t - p * nxh;
        const C zk = Z[p * nx + k];
        const C zm = Z[p * nx + (k == 0 ? 0 : nx - k)];
        const int q0 = 2 * p, q1 = 2 * p + 1;
        spec[q0 / R][(size_t)(line0 + q0 % R) * ldh + k] = mkc<T>((T)0.5 * (zk.x + zm.x), (T)0.5 * (zk.y - zm.y));
        spec[q1 / R][(size_t)(line0 + q1 % R) * ldh + k] = mkc<T>((T)0.5 * (zk.y + zm.y), (T)0.5 * (zm.x - zk.x));
    }
}

// Forward sensor sampling s = M p (Sec. III, M w; Sec. VI.A linear interpolation) for the rows
// of this CTA: p of row r is item r of `buf`.  One atomic add per (line, sensor) segment.
template <typename T>
__device__ void gather_rows(const DevPlan<T>& P, cplx<T>* buf, int line0, int R, T* data_row) {
    const DevSensors<T>& S = P.sens;
    const int s0 = S.g_lineptr[line0], s1 = S.g_lineptr[line0 + R];
    for (int s = s0 + (int)threadIdx.x; s < s1; s += blockDim.x) {
        const int r = S.g_seg_line[s] - line0;
        T acc = 0;
        for (int e = S.g_seg_e0[s]; e < S.g_seg_e0[s + 1]; ++e) acc += S.g_ent_w[e] * slot(buf, r, S.g_ent_x[e], P.nx);
        atomicAdd(&data_row[S.g_seg_sensor[s]], acc);
    }
}

// Adjoint injection p_bar += M^T h^n (the residual enters as a source, Sec. III Eq. (massa)).
// Segments are distinct grid points, so no two threads touch the same element.
template <typename T>
__device__ void scatter_rows(const DevPlan<T>& P, cplx<T>* buf, int line0, int R, const T* h_row) {
    const DevSensors<T>& S = P.sens;
    const int s0 = S.s_lineptr[line0], s1 = S.s_lineptr[line0 + R];
    for (int s = s0 + (int)threadIdx.x; s < s1; s += blockDim.x) {
        const int r = S.s_seg_line[s] - line0;
        T acc = 0;
        for (int e = S.s_seg_e0[s]; e < S.s_seg_e0[s + 1]; ++e) acc += S.s_ent_w[e] * h_row[S.s_ent_sensor[e]];
        slot(buf, r, S.s_seg_x[s], P.nx) += acc;
    }
}

template <typename T> __device__ __forceinline__ T pml_at(const T* const* tab, int xi, int i, int y, int z) {
    return xi == 0 ? tab[0][i] : (xi == 1 ? tab[1][y] : tab[2][z]);
}

struct RowSmem {
    template <typename T> __device__ static void carve(int nx, int qmax, cplx<T>*& tw, cplx<T>*& A, cplx<T>*& B) {
        extern __shared__ __align__(16) unsigned char smem_raw[];
        tw = reinterpret_cast<cplx<T>*>(smem_raw);
        A = tw + nx;
        B = A + (size_t)qmax * nx;
    }
};

// ------------------------------------------------------------------------------------------
// Forward row kernels
// ------------------------------------------------------------------------------------------

// Initial state (p^0 = p0, rho_xi^0 = p0 / (d c0^2)), sample s^0 = M p0, x-FFT of p0.
template <typename T, int D>
__global__ void k_fwd_init(DevPlan<T> P, int R, int last) {
    cplx<T>*tw, *A, *B;
    RowSmem::carve<T>(P.nx, R / 2, tw, A, B);
    const int nx = P.nx, line0 = blockIdx.x * R;
    load_tw(tw, P.twx, nx);
    for (int t = threadIdx.x; t < R * nx; t += blockDim.x) {
        const int r = t / nx, i = t - r * nx;
        const size_t idx = (size_t)(line0 + r) * nx + i;
        const T p = P.img[idx];
        const T rh = p / (T(D) * P.c2[idx]);
#pragma unroll
        for (int xi = 0; xi < D; ++xi) P.rh[xi][idx] = rh;
        slot(A, r, i, nx) = p;
    }
    __syncthreads();
    gather_rows(P, A, line0, R, P.data);
    if (last) return;
    __syncthreads();
    cplx<T>* res = fft_lines<T, false>(A, B, P.fx, tw, R / 2, 1, nx, false);
    r2c_unpack(res, P.spec, 1, R, line0, nx, P.ldh);
}

// u_xi^{n+1/2} = au (au u_xi^{n-1/2} - dt b_xi g_xi) with g_xi from spectra 0..d-1; on the first
// step u^{-1/2} = (dt/2) b_xi g_xi.  Then x-FFT of u_xi.
template <typename T, int D>
__global__ void k_fwd_u(DevPlan<T> P, int R, int first) {
    cplx<T>*tw, *A, *B;
    RowSmem::carve<T>(P.nx, D * R / 2, tw, A, B);
    const int nx = P.nx, line0 = blockIdx.x * R, Q = D * R / 2;
    load_tw(tw, P.twx, nx);
    c2r_pack(A, P.spec, D, R, line0, nx, P.ldh);
    __syncthreads();
    cplx<T>* res = fft_lines<T, true>(A, B, P.fx, tw, Q, 1, nx, false);
    cplx<T>* out = (res == A) ? B : A;
    const T dt = P.dt;
    for (int t = threadIdx.x; t < R * nx; t += blockDim.x) {
        const int r = t / nx, i = t - r * nx;
        const int line = line0 + r, y = line % P.ny, z = line / P.ny;
        const size_t idx = (size_t)line * nx + i;
#pragma unroll
        for (int xi = 0; xi < D; ++xi) {
            const T g = slot(res, xi * R + r, i, nx);
            const T bb = P.b[xi][idx];
            const T au = pml_at(P.au, xi, i, y, z);
            const T uo = first ? (T)0.5 * dt * bb * g : P.u[xi][idx];
            const T un = au * (au * uo - dt * bb * g);
            P.u[xi][idx] = un;
            slot(out, xi * R + r, i, nx) = un;
        }
    }
    __syncthreads();
    res = fft_lines<T, false>(out, res, P.fx, tw, Q, 1, nx, false);
    r2c_unpack(res, P.spec, D, R, line0, nx, P.ldh);
}

// rho_xi^{n+1} = a (a rho_xi^n - dt rho0 e_xi); dd = rho0 sum e; r = sum rho.  Lossless: p = c0^2 r,
// sample, x-FFT of p.  Lossy: keep r, x-FFT of (dd, r) for the fractional Laplacians.
template <typename T, int D>
__global__ void k_fwd_rho(DevPlan<T> P, int R, int last, T* data_row) {
    cplx<T>*tw, *A, *B;
    RowSmem::carve<T>(P.nx, D * R / 2, tw, A, B);
    const int nx = P.nx, line0 = blockIdx.x * R;
    load_tw(tw, P.twx, nx);
    c2r_pack(A, P.spec, D, R, line0, nx, P.ldh);
    __syncthreads();
    cplx<T>* res = fft_lines<T, true>(A, B, P.fx, tw, D * R / 2, 1, nx, false);
    cplx<T>* out = (res == A) ? B : A;
    const T dt = P.dt;
    for (int t = threadIdx.x; t < R * nx; t += blockDim.x) {
        const int r = t / nx, i = t - r * nx;
        const int line = line0 + r, y = line % P.ny, z = line / P.ny;
        const size_t idx = (size_t)line * nx + i;
        const T rho0 = P.rho0[idx];
        T rs = 0, es = 0;
#pragma unroll
        for (int xi = 0; xi < D; ++xi) {
            const T e = slot(res, xi * R + r, i, nx);
            const T a = pml_at(P.a, xi, i, y, z);
            const T rh = a * (a * P.rh[xi][idx] - dt * rho0 * e);
            P.rh[xi][idx] = rh;
            rs += rh;
            es += e;
        }
        if (P.lossy) {
            P.rsum[idx] = rs;
            slot(out, r, i, nx) = rho0 * es;
            slot(out, R + r, i, nx) = rs;
        } else {
            slot(out, r, i, nx) = P.c2[idx] * rs;
        }
    }
    __syncthreads();
    if (!P.lossy) {
        gather_rows(P, out, line0, R, data_row);
        if (last) return;
        __syncthreads();
    }
    const int F = P.lossy ? 2 : 1;
    res = fft_lines<T, false>(out, res, P.fx, tw, F * R / 2, 1, nx, false);
    r2c_unpack(res, P.spec, F, R, line0, nx, P.ldh);
}

// Lossy equation of state p = c0^2 r + c0^2 tau L_{y-2} dd - c0^2 eta L_{y-1} r (Eq. (state)),
// sample, x-FFT of p.
template <typename T, int D>
__global__ void k_fwd_p(DevPlan<T> P, int R, int last, T* data_row) {
    cplx<T>*tw, *A, *B;
    RowSmem::carve<T>(P.nx, R, tw, A, B);
    const int nx = P.nx, line0 = blockIdx.x * R;
    load_tw(tw, P.twx, nx);
    c2r_pack(A, P.spec, 2, R, line0, nx, P.ldh);
    __syncthreads();
    cplx<T>* res = fft_lines<T, true>(A, B, P.fx, tw, R, 1, nx, false);
    cplx<T>* out = (res == A) ? B : A;
    for (int t = threadIdx.x; t < R * nx; t += blockDim.x) {
        const int r = t / nx, i = t - r * nx;
        const size_t idx = (size_t)(line0 + r) * nx + i;
        const T Ld = slot(res, r, i, nx);
        const T Lr = slot(res, R + r, i, nx);
        slot(out, r, i, nx) = P.c2[idx] * P.rsum[idx] + P.c2tau[idx] * Ld - P.c2eta[idx] * Lr;
    }
    __syncthreads();
    gather_rows(P, out, line0, R, data_row);
    if (last) return;
    __syncthreads();
    res = fft_lines<T, false>(out, res, P.fx, tw, R / 2, 1, nx, false);
    r2c_unpack(res, P.spec, 1, R, line0, nx, P.ldh);
}

// ------------------------------------------------------------------------------------------
// Adjoint row kernels (exact transpose, reverse time)
// ------------------------------------------------------------------------------------------

// Shared tail once p_bar of a time level is known (items 0..R-1 of `pb`):
//   final: grad = p_bar + sum_xi rho_bar_xi / (d c0^2)   (transpose of the initial state)
//   lossy: keep p_bar; x-FFT of (c0^2 tau p_bar, c0^2 eta p_bar)
//   lossless: rho_bar_xi += c0^2 p_bar; e_bar_xi = -dt rho0 a rho_bar_xi; rho_bar_xi *= a^2;
//             x-FFT of e_bar_xi
template <typename T, int D>
__device__ void adj_tail(const DevPlan<T>& P, cplx<T>* pb, cplx<T>* other, const cplx<T>* tw, int line0, int R,
                         int final_) {
    const int nx = P.nx;
    const T dt = P.dt;
    if (final_) {
        for (int t = threadIdx.x; t < R * nx; t += blockDim.x) {
            const int r = t / nx, i = t - r * nx;
            const size_t idx = (size_t)(line0 + r) * nx + i;
            T s = 0;
#pragma unroll
            for (int xi = 0; xi < D; ++xi) s += P.rh[xi][idx];
            P.img[idx] = slot(pb, r, i, nx) + s / (T(D) * P.c2[idx]);
        }
        return;
    }
    for (int t = threadIdx.x; t < R * nx; t += blockDim.x) {
        const int r = t / nx, i = t - r * nx;
        const int line = line0 + r, y = line % P.ny, z = line / P.ny;
        const size_t idx = (size_t)line * nx + i;
        const T pv = slot(pb, r, i, nx);
        if (P.lossy) {
            P.pbar[idx] = pv;
            slot(other, r, i, nx) = P.c2tau[idx] * pv;
            slot(other, R + r, i, nx) = P.c2eta[idx] * pv;
        } else {
            const T rbar = P.c2[idx] * pv;
            const T rho0 = P.rho0[idx];
#pragma unroll
            for (int xi = 0; xi < D; ++xi) {
                const T a = pml_at(P.a, xi, i, y, z);
                const T rb = P.rh[xi][idx] + rbar;
                slot(other, xi * R + r, i, nx) = -dt * rho0 * a * rb;
                P.rh[xi][idx] = a * a * rb;
            }
        }
    }
    __syncthreads();
    const int F = P.lossy ? 2 : D;
    cplx<T>* res = fft_lines<T, false>(other, pb, P.fx, tw, F * R / 2, 1, nx, false);
    r2c_unpack(res, P.spec, F, R, line0, nx, P.ldh);
}

// p_bar^{Nt-1} = M^T h^{Nt-1}, then the tail.
template <typename T, int D>
__global__ void k_adj_init(DevPlan<T> P, int R, int final_, const T* h_row) {
    cplx<T>*tw, *A, *B;
    RowSmem::carve<T>(P.nx, (D > 2 ? D : 2) * R / 2, tw, A, B);
    const int nx = P.nx, line0 = blockIdx.x * R;
    load_tw(tw, P.twx, nx);
    for (int t = threadIdx.x; t < R * nx; t += blockDim.x) slot(A, t / nx, t % nx, nx) = 0;
    __syncthreads();
    scatter_rows(P, A, line0, R, h_row);
    __syncthreads();
    adj_tail<T, D>(P, A, B, tw, line0, R, final_);
}

// Lossy: r_bar = c0^2 p_bar - L_{y-1}(c0^2 eta p_bar), dd_bar = L_{y-2}(c0^2 tau p_bar);
// rho_bar_xi += r_bar; e_bar_xi = rho0 dd_bar - dt rho0 a rho_bar_xi; rho_bar_xi *= a^2; x-FFT e_bar.
template <typename T, int D>
__global__ void k_adj_rho(DevPlan<T> P, int R) {
    cplx<T>*tw, *A, *B;
    RowSmem::carve<T>(P.nx, (D > 2 ? D : 2) * R / 2, tw, A, B);
    const int nx = P.nx, line0 = blockIdx.x * R;
    load_tw(tw, P.twx, nx);
    c2r_pack(A, P.spec, 2, R, line0, nx, P.ldh);
    __syncthreads();
    cplx<T>* res = fft_lines<T, true>(A, B, P.fx, tw, R, 1, nx, false);
    cplx<T>* out = (res == A) ? B : A;
    const T dt = P.dt;
    for (int t = threadIdx.x; t < R * nx; t += blockDim.x) {
        const int r = t / nx, i = t - r * nx;
        const int line = line0 + r, y = line % P.ny, z = line / P.ny;
        const size_t idx = (size_t)line * nx + i;
        const T ddbar = slot(res, r, i, nx);
        const T w = slot(res, R + r, i, nx);
        const T rbar = P.c2[idx] * P.pbar[idx] - w;
        const T rho0 = P.rho0[idx];
        // e_bar values go to `out`; res items are consumed per point before being overwritten
#pragma unroll
        for (int xi = 0; xi < D; ++xi) {
            const T a = pml_at(P.a, xi, i, y, z);
            const T rb = P.rh[xi][idx] + rbar;
            slot(out, xi * R + r, i, nx) = rho0 * ddbar - dt * rho0 * a * rb;
            P.rh[xi][idx] = a * a * rb;
        }
    }
    __syncthreads();
    res = fft_lines<T, false>(out, res, P.fx, tw, D * R / 2, 1, nx, false);
    r2c_unpack(res, P.spec, D, R, line0, nx, P.ldh);
}

// u_bar_xi += (-D+ e_bar_xi); g_bar_xi = -dt b au u_bar_xi; u_bar_xi *= au^2; on the last reverse
// step the transpose of u^{-1/2} = (dt/2) b D+ p0 adds (dt/2) b u_bar_xi.  x-FFT of g_bar.
template <typename T, int D>
__global__ void k_adj_u(DevPlan<T> P, int R, int final_) {
    cplx<T>*tw, *A, *B;
    RowSmem::carve<T>(P.nx, D * R / 2, tw, A, B);
    const int nx = P.nx, line0 = blockIdx.x * R, Q = D * R / 2;
    load_tw(tw, P.twx, nx);
    c2r_pack(A, P.spec, D, R, line0, nx, P.ldh);
    __syncthreads();
    cplx<T>* res = fft_lines<T, true>(A, B, P.fx, tw, Q, 1, nx, false);
    cplx<T>* out = (res == A) ? B : A;
    const T dt = P.dt;
    for (int t = threadIdx.x; t < R * nx; t += blockDim.x) {
        const int r = t / nx, i = t - r * nx;
        const int line = line0 + r, y = line % P.ny, z = line / P.ny;
        const size_t idx = (size_t)line * nx + i;
#pragma unroll
        for (int xi = 0; xi < D; ++xi) {
            const T bb = P.b[xi][idx];
            const T au = pml_at(P.au, xi, i, y, z);
            T ub = P.u[xi][idx] + slot(res, xi * R + r, i, nx);
            T g = -dt * bb * au * ub;
            ub = au * au * ub;
            if (final_) g += (T)0.5 * dt * bb * ub;
            P.u[xi][idx] = ub;
            slot(out, xi * R + r, i, nx) = g;
        }
    }
    __syncthreads();
    res = fft_lines<T, false>(out, res, P.fx, tw, Q, 1, nx, false);
    r2c_unpack(res, P.spec, D, R, line0, nx, P.ldh);
}

// p_bar^n = -sum_xi D-_xi g_bar_xi (spectrum 0) + M^T h^n, then the tail.
template <typename T, int D>
__global__ void k_adj_p(DevPlan<T> P, int R, int final_, const T* h_row) {
    cplx<T>*tw, *A, *B;
    RowSmem::carve<T>(P.nx, (D > 2 ? D : 2) * R / 2, tw, A, B);
    const int nx = P.nx, line0 = blockIdx.x * R;
    load_tw(tw, P.twx, nx);
    c2r_pack(A, P.spec, 1, R, line0, nx, P.ldh);
    __syncthreads();
    cplx<T>* res = fft_lines<T, true>(A, B, P.fx, tw, R / 2, 1, nx, false);
    cplx<T>* other = (res == A) ? B : A;
    scatter_rows(P, res, line0, R, h_row);
    __syncthreads();
    adj_tail<T, D>(P, res, other, tw, line0, R, final_);
}

// ------------------------------------------------------------------------------------------
// Spectral kernels: transforms along y (lax = 1) or z (lax = 2) of half-spectrum columns,
// with the k-space multiply fused in between for the multiply modes.
// blockIdx.x = tile of W columns kx; blockIdx.y = outer index (z for lax = 1, y for lax = 2).
// ------------------------------------------------------------------------------------------
template <typename T, int D>
__device__ __forceinline__ cplx<T> spec_symbol(const DevPlan<T>& P, int mode, int f, int kx, int ky, int kz) {
    const size_t kidx = ((size_t)kz * P.ny + ky) * P.nxh + kx;
    if (mode == SPEC_ABS) {
        const T s = (f == 0) ? P.kpa[kidx] : P.kpb[kidx];
        return mkc<T>(s, 0);
    }
    const int kf = (f == 0) ? kx : (f == 1 ? ky : kz);
    const T kap = P.kapN[kidx];
    cplx<T> m = (mode == SPEC_GRAD || mode == SPEC_DIVT) ? P.dp[f][kf] : P.dm[f][kf];
    const T s = (mode == SPEC_DIVT || mode == SPEC_GRADT) ? -kap : kap;
    return cscale(m, s);
}

template <typename T, int D, int MODE>
__global__ void k_spec(DevPlan<T> P, int W, int lax, int F) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int L = (lax == 1) ? P.ny : P.nz;
    cplx<T>* tw = reinterpret_cast<cplx<T>*>(smem_raw);
    cplx<T>* X = tw + L;
    cplx<T>* Y = X + (size_t)L * W;
    cplx<T>* Z = Y + (size_t)L * W;
    const FftAxis& ax = (lax == 1) ? P.fy : P.fz;
    load_tw(tw, (lax == 1) ? P.twy : P.twz, L);

    const int kx0 = blockIdx.x * W;
    const int wv = min(W, P.nxh - kx0);
    const int outer = blockIdx.y;
    const size_t es = (lax == 1) ? (size_t)P.ldh : (size_t)P.ny * P.ldh;
    const size_t base = (lax == 1) ? (size_t)outer * P.ny * P.ldh + kx0 : (size_t)outer * P.ldh + kx0;
    const int total = L * W;

    auto load = [&](cplx<T>* buf, int f) {
        const cplx<T>* src = P.spec[f] + base;
        for (int t = threadIdx.x; t < total; t += blockDim.x) {
            const int i = t / W, c = t - i * W;
            buf[t] = (c < wv) ? src[(size_t)i * es + c] : mkc<T>(0, 0);
        }
    };
    auto store = [&](const cplx<T>* buf, int f) {
        cplx<T>* dst = P.spec[f] + base;
        for (int t = threadIdx.x; t < total; t += blockDim.x) {
            const int i = t / W, c = t - i * W;
            if (c < wv) dst[(size_t)i * es + c] = buf[t];
        }
    };
    // spectral indices of element (i, c): kx = kx0 + c; (ky, kz) = (i, outer) or (outer, i)
    auto symbol = [&](int mode, int f, int t) {
        const int i = t / W, c = t - i * W;
        const int ky = (lax == 1) ? i : outer;
        const int kz = (lax == 1) ? outer : i;
        return spec_symbol<T, D>(P, mode, f, kx0 + c < P.nxh ? kx0 + c : 0, ky, kz);
    };

    if (MODE == SPEC_PLAIN_FWD || MODE == SPEC_PLAIN_INV) {
        for (int f = 0; f < F; ++f) {
            load(X, f);
            __syncthreads();
            cplx<T>* r = (MODE == SPEC_PLAIN_FWD) ? fft_lines<T, false>(X, Y, ax, tw, W, W, 1, true)
                                                  : fft_lines<T, true>(X, Y, ax, tw, W, W, 1, true);
            store(r, f);
            __syncthreads();
        }
        return;
    }
    if (MODE == SPEC_GRAD) {
        load(X, 0);
        __syncthreads();
        cplx<T>* res = fft_lines<T, false>(X, Y, ax, tw, W, W, 1, true);
        cplx<T>* scr = (res == X) ? Y : X;
        for (int f = 0; f < D; ++f) {
            for (int t = threadIdx.x; t < total; t += blockDim.x) Z[t] = cmul(res[t], symbol(SPEC_GRAD, f, t));
            __syncthreads();
            cplx<T>* r = fft_lines<T, true>(Z, scr, ax, tw, W, W, 1, true);
            store(r, f);
            __syncthreads();
        }
        return;
    }
    if (MODE == SPEC_GRADT) {
        for (int f = 0; f < D; ++f) {
            load(X, f);
            __syncthreads();
            cplx<T>* res = fft_lines<T, false>(X, Y, ax, tw, W, W, 1, true);
            for (int t = threadIdx.x; t < total; t += blockDim.x) {
                const cplx<T> v = cmul(res[t], symbol(SPEC_GRADT, f, t));
                Z[t] = (f == 0) ? v : cadd(Z[t], v);
            }
            __syncthreads();
        }
        cplx<T>* r = fft_lines<T, true>(Z, X, ax, tw, W, W, 1, true);
        store(r, 0);
        return;
    }
    // SPEC_DIV, SPEC_DIVT, SPEC_ABS: field f -> field f with its own symbol
    const int nf = (MODE == SPEC_ABS) ? 2 : D;
    for (int f = 0; f < nf; ++f) {
        load(X, f);
        __syncthreads();
        cplx<T>* res = fft_lines<T, false>(X, Y, ax, tw, W, W, 1, true);
        for (int t = threadIdx.x; t < total; t += blockDim.x) res[t] = cmul(res[t], symbol(MODE, f, t));
        __syncthreads();
        cplx<T>* r = fft_lines<T, true>(res, (res == X) ? Y : X, ax, tw, W, W, 1, true);
        store(r, f);
        __syncthreads();
    }
}

}  // namespace pat
