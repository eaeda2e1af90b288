// pat_kernels.cuh -- the time-stepping kernels of the forward operator and its transpose.
//
// One time step of the k-space scheme (Sec. II.A) needs three spectral operations:
//   (1) g_xi = D+_xi p            (staggered gradient, momentum equation Eq. (mom))
//   (2) e_xi = D-_xi u_xi         (staggered divergence, mass equation Eq. (mass))
//   (3) L_{y-2} dd, L_{y-1} r     (fractional Laplacians of Eq. (state); lossy media only)
// Each spectral operation is  x-FFT -> [y-FFT -> multiply -> y-IFFT] -> x-IFFT.  The x
// transforms run in "row" kernels, where the pointwise physics of the step is fused between
// the inverse transform of one operation and the forward transform of the next, so every
// state field is read and written once per step.  The middle part runs in "spectral" kernels
// over tiles of half-spectrum columns.  Two real lines share one complex transform.
//
// Latency structure of every kernel:
//   prologue   constant operands (twiddles, medium rows, PML factors, symbol tables, sensor
//              lists) are staged into shared memory with cp.async before griddepcontrol.wait, so
//              under programmatic dependent launch they overlap the previous kernel;
//   main load  operands produced by earlier kernels (spectra, state rows) are staged with
//              cp.async right after the wait, all in flight at once;
//   compute    FFTs and physics out of shared memory; results stored straight to global.
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

// ------------------------------------------------------------------------------------------
// asynchronous copies and programmatic dependent launch
// ------------------------------------------------------------------------------------------
template <int BYTES> __device__ __forceinline__ void cp_async(void* s, const void* g) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(s);
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(g) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(g), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// contiguous block, 16-byte aligned at both ends, size a multiple of 16
__device__ __forceinline__ void stage16(void* s, const void* g, size_t bytes) {
    const int n16 = (int)(bytes >> 4);
    for (int k = threadIdx.x; k < n16; k += blockDim.x)
        cp_async<16>(static_cast<char*>(s) + 16 * (size_t)k, static_cast<const char*>(g) + 16 * (size_t)k);
}
// n elements of T, any alignment of T
template <typename T> __device__ __forceinline__ void stage_elems(T* s, const T* g, int n) {
    for (int k = threadIdx.x; k < n; k += blockDim.x) cp_async<sizeof(T)>(s + k, g + k);
}

// ------------------------------------------------------------------------------------------
// tensor memory access (cp.async.bulk.tensor) with an mbarrier that counts the bytes in flight
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(a), "r"(count) : "memory");
    // make the initialised barrier visible to the asynchronous (tensor-copy) proxy
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(a), "r"(bytes) : "memory");
}
// box of a 3-D tensor map at coordinates (c0, c1, c2) into shared memory, completing on `bar`
__device__ __forceinline__ void tma_load_3d(void* dst, const void* tmap, int c0, int c1, int c2,
                                            unsigned long long* bar) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const unsigned b = (unsigned)__cvta_generic_to_shared(bar);
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(d),
        "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(b)
        : "memory");
}
// wait for phase `parity` of the barrier to complete, at most `tries` polls; true when it did
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, unsigned tries) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
    for (unsigned k = 0; k < tries; ++k) {
        unsigned done = 0;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Wait for the preceding kernel of the stream (and its memory) -- a no-op without PDL.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
// Let the next kernel of the stream start its prologue.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

// real value of item q (= field * rows + row) at position i: items 2p, 2p+1 share complex line p
template <typename C> __device__ __forceinline__ auto& slot(C* buf, int q, int i, int nx) {
    C& c = buf[(q >> 1) * nx + i];
    return (q & 1) ? c.y : c.x;
}

// ------------------------------------------------------------------------------------------
// row kernels: shared-memory layout
// ------------------------------------------------------------------------------------------
constexpr int kSegCap = 1024;   // sensor segments per CTA staged in shared memory

template <int D> struct RowDims {
    static constexpr int FMAX = (D > 2 ? D : 2);   // spectra in or out of one row kernel
    static constexpr int NFMAX = 2 * D + 2;        // staged real field rows
};

// tw[nx] | A[qmax nx] | B[qmax nx] | S[FMAX R ldh] (complex) | F[NFMAX R nx] | pml[nx + 2R]
// (real, padded to 4) | seg_i[2 kSegCap] (int) | seg_w[2 kSegCap] (real)
template <typename T, int D> struct RowSm {
    cplx<T>* tw;
    cplx<T>* A;
    cplx<T>* B;
    cplx<T>* S;
    T* F;
    T* pml;
    int* seg_i;
    T* seg_w;
    int nx, R;
    __device__ RowSm(int nx_, int ldh, int R_) : nx(nx_), R(R_) {
        extern __shared__ __align__(16) unsigned char smem_raw[];
        const int qmax = RowDims<D>::FMAX * R / 2;
        tw = reinterpret_cast<cplx<T>*>(smem_raw);
        A = tw + nx;
        B = A + (size_t)qmax * nx;
        S = B + (size_t)qmax * nx;
        F = reinterpret_cast<T*>(S + (size_t)RowDims<D>::FMAX * R * ldh);
        pml = F + (size_t)RowDims<D>::NFMAX * R * nx;
        seg_w = pml + ((nx + 2 * R + 3) & ~3);
        seg_i = reinterpret_cast<int*>(seg_w + 2 * kSegCap);
    }
    __device__ T* row(int j) const { return F + (size_t)j * R * nx; }
    // PML factor of axis xi at (row r, x = i)
    __device__ T pml_at(int xi, int r, int i) const { return xi == 0 ? pml[i] : pml[nx + (xi - 1) * R + r]; }
};

template <typename T> size_t row_smem_bytes(int D, int nx, int ldh, int R) {
    const int fmax = D > 2 ? D : 2, nfmax = 2 * D + 2, qmax = fmax * R / 2;
    size_t b = (size_t)(nx + 2 * qmax * nx + fmax * R * ldh) * sizeof(cplx<T>);
    b += (size_t)(nfmax * R * nx + ((nx + 2 * R + 3) & ~3) + 2 * kSegCap) * sizeof(T);
    b += (size_t)2 * kSegCap * sizeof(int);
    return b;
}

// stage `R` consecutive x-lines of a real field (contiguous block)
template <typename T> __device__ __forceinline__ void stage_rows(T* dst, const T* field, int line0, int R, int nx) {
    stage16(dst, field + (size_t)line0 * nx, (size_t)R * nx * sizeof(T));
}

// stage F half spectra (R lines each) into S: item q = f R + r lands at S + q ldh
template <typename C>
__device__ __forceinline__ void stage_spectra(C* S, C* const* spec, int F, int line0, int R, int ldh) {
    for (int f = 0; f < F; ++f)
        stage16(S + (size_t)f * R * ldh, spec[f] + (size_t)line0 * ldh, (size_t)R * ldh * sizeof(C));
}

// PML factors of this CTA: the x table, and the y / z values of its R lines
template <typename T, int D>
__device__ __forceinline__ void stage_pml(const RowSm<T, D>& sm, const T* const* tab, const DevPlan<T>& P, int line0) {
    stage_elems(sm.pml, tab[0], P.nx);
    for (int t = threadIdx.x; t < (D - 1) * sm.R; t += blockDim.x) {
        const int ax = 1 + t / sm.R, r = t - (ax - 1) * sm.R;
        const int line = line0 + r;
        const int idx = (ax == 1) ? line % P.ny : line / P.ny;
        sm.pml[P.nx + t] = tab[ax][idx];
    }
}

// Pack F staged half spectra (item q at S + q ldh) into Q = F R / 2 complex lines so that one
// inverse transform per line yields two real lines (C2R of two Hermitian half spectra).
template <typename C>
__device__ void c2r_pack(C* Z, const C* S, int F, int R, int nx, int ldh) {
    using T = decltype(Z->x);
    const int nxh = nx / 2 + 1, Q = F * R / 2, half = nx / 2;
    for (int p = 0; p < Q; ++p)
    for (int k = threadIdx.x; k < nxh; k += blockDim.x) {
        C A = S[(size_t)(2 * p) * ldh + k];
        C B = S[(size_t)(2 * p + 1) * ldh + k];
        if (k == 0 || k == half) {
            A.y = 0;
            B.y = 0;
        }
        Z[p * nx + k] = mkc<T>(A.x - B.y, A.y + B.x);                              // A + i B
        if (k > 0 && k < half) Z[p * nx + nx - k] = mkc<T>(A.x + B.y, B.x - A.y);  // conj(A) + i conj(B)
    }
}

// Split Q forward-transformed complex lines (two real lines each) into F half spectra.
template <typename C>
__device__ void r2c_unpack(const C* Z, C* const* spec, int F, int R, int line0, int nx, int ldh) {
    using T = decltype(Z->x);
    const int nxh = nx / 2 + 1, Q = F * R / 2;
    for (int p = 0; p < Q; ++p)
    for (int k = threadIdx.x; k < nxh; k += blockDim.x) {
        const C zk = Z[p * nx + k];
        const C zm = Z[p * nx + (k == 0 ? 0 : nx - k)];
        const int q0 = 2 * p, q1 = 2 * p + 1;
        spec[q0 / R][(size_t)(line0 + q0 % R) * ldh + k] = mkc<T>((T)0.5 * (zk.x + zm.x), (T)0.5 * (zk.y - zm.y));
        spec[q1 / R][(size_t)(line0 + q1 % R) * ldh + k] = mkc<T>((T)0.5 * (zk.y + zm.y), (T)0.5 * (zm.x - zk.x));
    }
}

// ------------------------------------------------------------------------------------------
// sensors (Sec. III: s = M p; the adjoint injects M^T h as a source, Eq. (massa))
// ------------------------------------------------------------------------------------------
// A gather segment is one (x-line, sensor) pair: weights w0 at x0 and w1 at x0 + 1 (w1 = 0 for
// a single entry).  seg_i holds (sensor, r * nx + x0) pairs, seg_w (w0, w1) pairs.
template <typename T, int D>
__device__ __forceinline__ int2 gather_prologue(const RowSm<T, D>& sm, const DevPlan<T>& P, int line0) {
    const DevSensors<T>& S = P.sens;
    const int s0 = S.g_lineptr[line0], s1 = S.g_lineptr[line0 + sm.R];
    const int n = min(s1 - s0, kSegCap);
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        sm.seg_i[2 * t] = S.g_seg_sensor[s0 + t];
        sm.seg_i[2 * t + 1] = (S.g_seg_line[s0 + t] - line0) * P.nx + S.g_seg_x0[s0 + t];
        sm.seg_w[2 * t] = S.g_seg_w0[s0 + t];
        sm.seg_w[2 * t + 1] = S.g_seg_w1[s0 + t];
    }
    return make_int2(s0, s1);
}

// s^n_j += this CTA's part of sensor j (pressure of row r = item r of `buf`).  One atomic add per
// (line, sensor) segment: a 2-D bilinear sensor receives two adds onto zero, order-independent.
template <typename T, int D>
__device__ void gather_rows(const RowSm<T, D>& sm, const DevPlan<T>& P, int2 rng, int line0, const cplx<T>* buf,
                            T* data_row) {
    const DevSensors<T>& S = P.sens;
    const int nx = P.nx;
    for (int t = threadIdx.x; t < rng.y - rng.x; t += blockDim.x) {
        int j, pos;
        T w0, w1;
        if (t < kSegCap) {
            j = sm.seg_i[2 * t];
            pos = sm.seg_i[2 * t + 1];
            w0 = sm.seg_w[2 * t];
            w1 = sm.seg_w[2 * t + 1];
        } else {
            const int s = rng.x + t;
            j = S.g_seg_sensor[s];
            pos = (S.g_seg_line[s] - line0) * nx + S.g_seg_x0[s];
            w0 = S.g_seg_w0[s];
            w1 = S.g_seg_w1[s];
        }
        const int r = pos / nx, x = pos - r * nx;
        T acc = w0 * slot(buf, r, x, nx);
        if (w1 != (T)0) acc += w1 * slot(buf, r, x + 1, nx);
        atomicAdd(&data_row[j], acc);
    }
}

// Adjoint injection, prologue part: for every grid point of this CTA that a sensor touches,
// v = sum_j w_j h_j (the residual record is read-only during the adjoint solve).  seg_i holds
// r * nx + x, seg_w the value.
template <typename T, int D>
__device__ __forceinline__ int2 scatter_prologue(const RowSm<T, D>& sm, const DevPlan<T>& P, int line0,
                                                  const T* h_row) {
    const DevSensors<T>& S = P.sens;
    const int s0 = S.s_lineptr[line0], s1 = S.s_lineptr[line0 + sm.R];
    const int n = min(s1 - s0, kSegCap);
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const int s = s0 + t;
        T acc = 0;
        for (int e = S.s_seg_e0[s]; e < S.s_seg_e0[s + 1]; ++e) acc += S.s_ent_w[e] * h_row[S.s_ent_sensor[e]];
        sm.seg_i[t] = (S.s_seg_line[s] - line0) * P.nx + S.s_seg_x[s];
        sm.seg_w[t] = acc;
    }
    return make_int2(s0, s1);
}

// p_bar += M^T h^n on this CTA's lines (items 0..R-1 of `buf`); segments are distinct points.
template <typename T, int D>
__device__ void scatter_rows(const RowSm<T, D>& sm, const DevPlan<T>& P, int2 rng, cplx<T>* buf, int line0,
                             const T* h_row) {
    const DevSensors<T>& S = P.sens;
    const int nx = P.nx;
    for (int t = threadIdx.x; t < rng.y - rng.x; t += blockDim.x) {
        int pos;
        T v;
        if (t < kSegCap) {
            pos = sm.seg_i[t];
            v = sm.seg_w[t];
        } else {
            const int s = rng.x + t;
            v = 0;
            for (int e = S.s_seg_e0[s]; e < S.s_seg_e0[s + 1]; ++e) v += S.s_ent_w[e] * h_row[S.s_ent_sensor[e]];
            pos = (S.s_seg_line[s] - line0) * nx + S.s_seg_x[s];
        }
        const int r = pos / nx, x = pos - r * nx;
        slot(buf, r, x, nx) += v;
    }
}

// ------------------------------------------------------------------------------------------
// Forward row kernels
// ------------------------------------------------------------------------------------------

// Initial state (p^0 = p0, rho_xi^0 = p0 / (d c0^2)), sample s^0 = M p0, x-FFT of p0.
template <typename T, int D>
__global__ void __launch_bounds__(256) k_fwd_init(DevPlan<T> P, int R, int last) {
    RowSm<T, D> sm(P.nx, P.ldh, R);
    const int nx = P.nx, line0 = blockIdx.x * R;
    stage16(sm.tw, P.twx, (size_t)nx * sizeof(cplx<T>));
    stage_rows(sm.row(0), P.c2, line0, R, nx);
    stage_rows(sm.row(1), P.img, line0, R, nx);
    cp_commit();
    const int2 g = gather_prologue(sm, P, line0);
    pdl_trigger();
    pdl_wait();
    cp_wait_all();
    __syncthreads();
    for (int r = 0; r < R; ++r)
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        const int t = r * nx + i;
        const size_t idx = (size_t)(line0 + r) * nx + i;
        const T p = sm.row(1)[t];
        const T rh = p / (T(D) * sm.row(0)[t]);
#pragma unroll
        for (int xi = 0; xi < D; ++xi) P.rh[xi][idx] = rh;
        slot(sm.A, r, i, nx) = p;
    }
    __syncthreads();
    gather_rows(sm, P, g, line0, sm.A, P.data);
    if (last) return;
    __syncthreads();
    cplx<T>* res = fft_rows<T, false>(sm.A, sm.B, P.fx, sm.tw, R / 2);
    r2c_unpack(res, P.spec, 1, R, line0, nx, P.ldh);
}

// u_xi^{n+1/2} = au (au u_xi^{n-1/2} - dt b_xi g_xi) with g_xi from spectra 0..d-1; on the first
// step u^{-1/2} = (dt/2) b_xi g_xi.  Then x-FFT of u_xi.
template <typename T, int D>
__global__ void __launch_bounds__(256) k_fwd_u(DevPlan<T> P, int R, int first) {
    RowSm<T, D> sm(P.nx, P.ldh, R);
    const int nx = P.nx, line0 = blockIdx.x * R, Q = D * R / 2;
    stage16(sm.tw, P.twx, (size_t)nx * sizeof(cplx<T>));
#pragma unroll
    for (int xi = 0; xi < D; ++xi) stage_rows(sm.row(xi), P.b[xi], line0, R, nx);
    stage_pml(sm, P.au, P, line0);
    cp_commit();
    pdl_trigger();
    pdl_wait();
    stage_spectra(sm.S, P.spec, D, line0, R, P.ldh);
    if (!first) {
#pragma unroll
        for (int xi = 0; xi < D; ++xi) stage_rows(sm.row(D + xi), P.u[xi], line0, R, nx);
    }
    cp_commit();
    cp_wait_all();
    __syncthreads();
    c2r_pack(sm.A, sm.S, D, R, nx, P.ldh);
    __syncthreads();
    cplx<T>* res = fft_rows<T, true>(sm.A, sm.B, P.fx, sm.tw, Q);
    cplx<T>* out = (res == sm.A) ? sm.B : sm.A;
    const T dt = P.dt;
    for (int r = 0; r < R; ++r)
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        const int t = r * nx + i;
        const size_t idx = (size_t)(line0 + r) * nx + i;
#pragma unroll
        for (int xi = 0; xi < D; ++xi) {
            const T g = slot(res, xi * R + r, i, nx);
            const T bb = sm.row(xi)[t];
            const T au = sm.pml_at(xi, r, i);
            const T uo = first ? (T)0.5 * dt * bb * g : sm.row(D + xi)[t];
            const T un = au * (au * uo - dt * bb * g);
            P.u[xi][idx] = un;
            slot(out, xi * R + r, i, nx) = un;
            if (P.hk_g[0]) P.hk_g[xi][idx] = g;
        }
    }
    __syncthreads();
    res = fft_rows<T, false>(out, res, P.fx, sm.tw, Q);
    r2c_unpack(res, P.spec, D, R, line0, nx, P.ldh);
}

// rho_xi^{n+1} = a (a rho_xi^n - dt rho0 e_xi); dd = rho0 sum e; r = sum rho.  Lossless: p = c0^2 r,
// sample, x-FFT of p.  Lossy: keep r, x-FFT of (dd, r) for the fractional Laplacians.
template <typename T, int D>
__global__ void __launch_bounds__(256) k_fwd_rho(DevPlan<T> P, int R, int last, T* data_row, T* qrow) {
    RowSm<T, D> sm(P.nx, P.ldh, R);
    const int nx = P.nx, line0 = blockIdx.x * R;
    stage16(sm.tw, P.twx, (size_t)nx * sizeof(cplx<T>));
    stage_rows(sm.row(0), P.rho0, line0, R, nx);
    if (!P.lossy) stage_rows(sm.row(1), P.c2, line0, R, nx);
    stage_pml(sm, P.a, P, line0);
    cp_commit();
    int2 g = make_int2(0, 0);
    if (P.atd) g = scatter_prologue(sm, P, line0, P.atd_row);
    else if (!P.lossy) g = gather_prologue(sm, P, line0);
    pdl_trigger();
    pdl_wait();
    stage_spectra(sm.S, P.spec, D, line0, R, P.ldh);
#pragma unroll
    for (int xi = 0; xi < D; ++xi) stage_rows(sm.row(2 + xi), P.rh[xi], line0, R, nx);
    cp_commit();
    cp_wait_all();
    __syncthreads();
    c2r_pack(sm.A, sm.S, D, R, nx, P.ldh);
    __syncthreads();
    cplx<T>* res = fft_rows<T, true>(sm.A, sm.B, P.fx, sm.tw, D * R / 2);
    cplx<T>* out = (res == sm.A) ? sm.B : sm.A;
    if (P.atd) {   // s = M^T atd_row into items 0 .. R-1 of `out`, read back by the pointwise step
        for (int q = threadIdx.x; q < (R / 2) * nx; q += blockDim.x) out[q] = mkc<T>(0, 0);
        __syncthreads();
        scatter_rows(sm, P, g, out, line0, P.atd_row);
        __syncthreads();
    }
    const T dt = P.dt;
    for (int r = 0; r < R; ++r)
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        const int t = r * nx + i;
        const size_t idx = (size_t)(line0 + r) * nx + i;
        const T rho0 = sm.row(0)[t];
        const T src = P.atd ? slot(out, r, i, nx) : (T)0;
        const int trj = P.tr_node ? P.tr_node[idx] : -1;
        T rs = 0, es = 0;
#pragma unroll
        for (int xi = 0; xi < D; ++xi) {
            const T e = slot(res, xi * R + r, i, nx);
            const T a = sm.pml_at(xi, r, i);
            const T rh = P.atd ? a * (a * sm.row(2 + xi)[t] - dt * rho0 * e + dt * rho0 * src / T(D))
                               : a * (a * sm.row(2 + xi)[t] - dt * rho0 * e);
            P.rh[xi][idx] = (trj >= 0) ? P.tr_row[trj] / (T(D) * P.c2[idx]) : rh;
            rs += rh;
            es += e;
            if (P.hk_e[0]) P.hk_e[xi][idx] = e;
        }
        if (P.lossy) {
            P.rsum[idx] = rs;
            if (P.atd) {
                slot(out, r, i, nx) = P.c2tau[idx] * (src - es);
                slot(out, R + r, i, nx) = P.c2eta[idx] * rs / rho0;
            } else {
                slot(out, r, i, nx) = rho0 * es;
                slot(out, R + r, i, nx) = rs;
            }
        } else {
            T pv = sm.row(1)[t] * rs;
            if (trj >= 0) pv = P.tr_row[trj];
            if (P.tr_img && last) P.tr_img[idx] = pv;
            slot(out, r, i, nx) = pv;
            if (qrow) qrow[idx] = rs;   // d p / d c0^2 (lossless)
        }
    }
    __syncthreads();
    if (!P.lossy) {
        if (!P.atd) gather_rows(sm, P, g, line0, out, data_row);
        if (last) return;
        __syncthreads();
    }
    const int F = P.lossy ? 2 : 1;
    res = fft_rows<T, false>(out, res, P.fx, sm.tw, F * R / 2);
    r2c_unpack(res, P.spec, F, R, line0, nx, P.ldh);
}

// Lossy equation of state p = c0^2 r + c0^2 tau L_{y-2} dd - c0^2 eta L_{y-1} r (Eq. (state)),
// sample, x-FFT of p.
template <typename T, int D>
__global__ void __launch_bounds__(256) k_fwd_p(DevPlan<T> P, int R, int last, T* data_row, T* qrow) {
    RowSm<T, D> sm(P.nx, P.ldh, R);
    const int nx = P.nx, line0 = blockIdx.x * R;
    stage16(sm.tw, P.twx, (size_t)nx * sizeof(cplx<T>));
    stage_rows(sm.row(0), P.c2, line0, R, nx);
    stage_rows(sm.row(1), P.c2tau, line0, R, nx);
    stage_rows(sm.row(2), P.c2eta, line0, R, nx);
    cp_commit();
    const int2 g = gather_prologue(sm, P, line0);
    pdl_trigger();
    pdl_wait();
    stage_spectra(sm.S, P.spec, 2, line0, R, P.ldh);
    stage_rows(sm.row(3), P.rsum, line0, R, nx);
    cp_commit();
    cp_wait_all();
    __syncthreads();
    c2r_pack(sm.A, sm.S, 2, R, nx, P.ldh);
    __syncthreads();
    cplx<T>* res = fft_rows<T, true>(sm.A, sm.B, P.fx, sm.tw, R);
    cplx<T>* out = (res == sm.A) ? sm.B : sm.A;
    for (int r = 0; r < R; ++r)
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        const int t = r * nx + i;
        const T Ld = slot(res, r, i, nx);
        const T Lr = slot(res, R + r, i, nx);
        const size_t idx = (size_t)(line0 + r) * nx + i;
        T pv;
        if (P.atd) {
            const T rho0 = P.rho0[idx];
            pv = sm.row(0)[t] * sm.row(3)[t] - rho0 * Ld - rho0 * Lr;
        } else {
            pv = sm.row(0)[t] * sm.row(3)[t] + sm.row(1)[t] * Ld - sm.row(2)[t] * Lr;
        }
        if (P.tr_node) {
            const int trj = P.tr_node[idx];
            if (trj >= 0) pv = P.tr_row[trj];
        }
        if (P.tr_img && last) P.tr_img[idx] = pv;
        slot(out, r, i, nx) = pv;
        if (qrow) {
            // d p / d c0^2 with tau, eta following c0 (Eq. (Twelve)): d(c0^2 tau)/d c0^2 = (y+1)/2 tau,
            // d(c0^2 eta)/d c0^2 = (y+2)/2 eta; (y+1)/2 = phb + 1, (y+2)/2 = pha + 2
            const T c2 = sm.row(0)[t];
            qrow[(size_t)(line0 + r) * nx + i] =
                sm.row(3)[t] + ((P.phb + (T)1) * sm.row(1)[t] * Ld - (P.pha + (T)2) * sm.row(2)[t] * Lr) / c2;
        }
    }
    __syncthreads();
    gather_rows(sm, P, g, line0, out, data_row);
    if (last) return;
    __syncthreads();
    res = fft_rows<T, false>(out, res, P.fx, sm.tw, R / 2);
    r2c_unpack(res, P.spec, 1, R, line0, nx, P.ldh);
}

// ------------------------------------------------------------------------------------------
// Adjoint row kernels (exact transpose, reverse time)
// ------------------------------------------------------------------------------------------

// Constant operands of the tail: lossy (not final) c0^2 tau, c0^2 eta in rows 0, 1; otherwise
// c0^2, rho0 in rows 0, 1 and the PML a.  The state rho_bar_xi goes to rows 2.. after the wait.
template <typename T, int D>
__device__ __forceinline__ void adj_tail_prologue(const RowSm<T, D>& sm, const DevPlan<T>& P, int line0,
                                                  int final_) {
    const int R = sm.R, nx = P.nx;
    if (P.lossy && !final_) {
        stage_rows(sm.row(0), P.c2tau, line0, R, nx);
        stage_rows(sm.row(1), P.c2eta, line0, R, nx);
    } else {
        stage_rows(sm.row(0), P.c2, line0, R, nx);
        stage_rows(sm.row(1), P.rho0, line0, R, nx);
        stage_pml(sm, P.a, P, line0);
    }
}
template <typename T, int D>
__device__ __forceinline__ void adj_tail_state(const RowSm<T, D>& sm, const DevPlan<T>& P, int line0, int final_) {
    if (P.lossy && !final_) return;
#pragma unroll
    for (int xi = 0; xi < D; ++xi) stage_rows(sm.row(2 + xi), P.rh[xi], line0, sm.R, P.nx);
}

// Shared tail once p_bar of a time level is known (items 0..R-1 of `pb`):
//   final: grad = p_bar + sum_xi rho_bar_xi / (d c0^2)   (transpose of the initial state)
//   lossy: keep p_bar; x-FFT of (c0^2 tau p_bar, c0^2 eta p_bar)
//   lossless: rho_bar_xi += c0^2 p_bar; e_bar_xi = -dt rho0 a rho_bar_xi; rho_bar_xi *= a^2;
//             x-FFT of e_bar_xi
//
// Medium gradient (optional, gc2 != nullptr): g_c2 += p_bar * q of this level (q = d p / d c0^2 of
// the recomputed forward, `qrow`), and at the final level the initial-density term
// g_c2 -= sum_xi rho_bar_xi p0 / (d c0^4) (rho_xi^0 = p0 / (d c0^2); p0 = `p0c`).
template <typename T, int D>
__device__ void adj_tail(const RowSm<T, D>& sm, const DevPlan<T>& P, cplx<T>* pb, cplx<T>* other, int line0,
                         int final_, const T* qrow = nullptr, T* gc2 = nullptr, const T* p0c = nullptr) {
    const int nx = P.nx, R = sm.R;
    const T dt = P.dt;
    if (final_) {
        for (int r = 0; r < R; ++r)
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            const int t = r * nx + i;
            const size_t idx = (size_t)(line0 + r) * nx + i;
            T s = 0;
#pragma unroll
            for (int xi = 0; xi < D; ++xi) s += sm.row(2 + xi)[t];
            const T c2 = sm.row(0)[t];
            P.img[idx] = slot(pb, r, i, nx) + s / (T(D) * c2);
            if (gc2) gc2[idx] -= s * p0c[idx] / (T(D) * c2 * c2);
        }
        return;
    }
    for (int r = 0; r < R; ++r)
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        const int t = r * nx + i;
        const size_t idx = (size_t)(line0 + r) * nx + i;
        const T pv = slot(pb, r, i, nx);
        if (gc2) gc2[idx] += pv * qrow[idx];
        if (P.lossy) {
            P.pbar[idx] = pv;
            slot(other, r, i, nx) = sm.row(0)[t] * pv;
            slot(other, R + r, i, nx) = sm.row(1)[t] * pv;
        } else {
            const T rbar = sm.row(0)[t] * pv;
            const T rho0 = sm.row(1)[t];
            T gr = 0;
#pragma unroll
            for (int xi = 0; xi < D; ++xi) {
                const T a = sm.pml_at(xi, r, i);
                const T rb = sm.row(2 + xi)[t] + rbar;
                slot(other, xi * R + r, i, nx) = -dt * rho0 * a * rb;
                P.rh[xi][idx] = a * a * rb;
                if (P.hk_grho) gr += P.hk_ein[xi][idx] * (-dt * a * rb);
            }
            if (P.hk_grho) P.hk_grho[idx] += gr;
        }
    }
    __syncthreads();
    const int F = P.lossy ? 2 : D;
    cplx<T>* res = fft_rows<T, false>(other, pb, P.fx, sm.tw, F * R / 2);
    r2c_unpack(res, P.spec, F, R, line0, nx, P.ldh);
}

// p_bar^{Nt-1} = M^T h^{Nt-1}, then the tail.
template <typename T, int D>
__global__ void __launch_bounds__(256) k_adj_init(DevPlan<T> P, int R, int final_, const T* h_row, const T* qrow,
                                                   T* gc2, const T* p0c) {
    RowSm<T, D> sm(P.nx, P.ldh, R);
    const int nx = P.nx, line0 = blockIdx.x * R;
    stage16(sm.tw, P.twx, (size_t)nx * sizeof(cplx<T>));
    adj_tail_prologue(sm, P, line0, final_);
    cp_commit();
    const int2 g = scatter_prologue(sm, P, line0, h_row);
    pdl_trigger();
    pdl_wait();
    adj_tail_state(sm, P, line0, final_);
    cp_commit();
    for (int r = 0; r < R; ++r)
        for (int i = threadIdx.x; i < nx; i += blockDim.x) slot(sm.A, r, i, nx) = 0;
    cp_wait_all();
    __syncthreads();
    scatter_rows(sm, P, g, sm.A, line0, h_row);
    __syncthreads();
    adj_tail(sm, P, sm.A, sm.B, line0, final_, qrow, gc2, p0c);
}

// Lossy: r_bar = c0^2 p_bar - L_{y-1}(c0^2 eta p_bar), dd_bar = L_{y-2}(c0^2 tau p_bar);
// rho_bar_xi += r_bar; e_bar_xi = rho0 dd_bar - dt rho0 a rho_bar_xi; rho_bar_xi *= a^2; x-FFT e_bar.
template <typename T, int D>
__global__ void __launch_bounds__(256) k_adj_rho(DevPlan<T> P, int R) {
    RowSm<T, D> sm(P.nx, P.ldh, R);
    const int nx = P.nx, line0 = blockIdx.x * R;
    stage16(sm.tw, P.twx, (size_t)nx * sizeof(cplx<T>));
    stage_rows(sm.row(0), P.c2, line0, R, nx);
    stage_rows(sm.row(1), P.rho0, line0, R, nx);
    stage_pml(sm, P.a, P, line0);
    cp_commit();
    pdl_trigger();
    pdl_wait();
    stage_spectra(sm.S, P.spec, 2, line0, R, P.ldh);
    stage_rows(sm.row(2), P.pbar, line0, R, nx);
#pragma unroll
    for (int xi = 0; xi < D; ++xi) stage_rows(sm.row(3 + xi), P.rh[xi], line0, R, nx);
    cp_commit();
    cp_wait_all();
    __syncthreads();
    c2r_pack(sm.A, sm.S, 2, R, nx, P.ldh);
    __syncthreads();
    cplx<T>* res = fft_rows<T, true>(sm.A, sm.B, P.fx, sm.tw, R);
    cplx<T>* out = (res == sm.A) ? sm.B : sm.A;
    const T dt = P.dt;
    for (int r = 0; r < R; ++r)
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        const int t = r * nx + i;
        const size_t idx = (size_t)(line0 + r) * nx + i;
        const T ddbar = slot(res, r, i, nx);
        const T w = slot(res, R + r, i, nx);
        const T rbar = sm.row(0)[t] * sm.row(2)[t] - w;
        const T rho0 = sm.row(1)[t];
        T gr = 0;
#pragma unroll
        for (int xi = 0; xi < D; ++xi) {
            const T a = sm.pml_at(xi, r, i);
            const T rb = sm.row(3 + xi)[t] + rbar;
            slot(out, xi * R + r, i, nx) = rho0 * ddbar - dt * rho0 * a * rb;
            P.rh[xi][idx] = a * a * rb;
            if (P.hk_grho) gr += P.hk_ein[xi][idx] * (ddbar - dt * a * rb);
        }
        if (P.hk_grho) P.hk_grho[idx] += gr;
    }
    __syncthreads();
    res = fft_rows<T, false>(out, res, P.fx, sm.tw, D * R / 2);
    r2c_unpack(res, P.spec, D, R, line0, nx, P.ldh);
}

// u_bar_xi += (-D+ e_bar_xi); g_bar_xi = -dt b au u_bar_xi; u_bar_xi *= au^2; on the last reverse
// step the transpose of u^{-1/2} = (dt/2) b D+ p0 adds (dt/2) b u_bar_xi.  x-FFT of g_bar.
template <typename T, int D>
__global__ void __launch_bounds__(256) k_adj_u(DevPlan<T> P, int R, int final_) {
    RowSm<T, D> sm(P.nx, P.ldh, R);
    const int nx = P.nx, line0 = blockIdx.x * R, Q = D * R / 2;
    stage16(sm.tw, P.twx, (size_t)nx * sizeof(cplx<T>));
#pragma unroll
    for (int xi = 0; xi < D; ++xi) stage_rows(sm.row(xi), P.b[xi], line0, R, nx);
    stage_pml(sm, P.au, P, line0);
    cp_commit();
    pdl_trigger();
    pdl_wait();
    stage_spectra(sm.S, P.spec, D, line0, R, P.ldh);
#pragma unroll
    for (int xi = 0; xi < D; ++xi) stage_rows(sm.row(D + xi), P.u[xi], line0, R, nx);
    cp_commit();
    cp_wait_all();
    __syncthreads();
    c2r_pack(sm.A, sm.S, D, R, nx, P.ldh);
    __syncthreads();
    cplx<T>* res = fft_rows<T, true>(sm.A, sm.B, P.fx, sm.tw, Q);
    cplx<T>* out = (res == sm.A) ? sm.B : sm.A;
    const T dt = P.dt;
    for (int r = 0; r < R; ++r)
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        const int t = r * nx + i;
        const size_t idx = (size_t)(line0 + r) * nx + i;
#pragma unroll
        for (int xi = 0; xi < D; ++xi) {
            const T bb = sm.row(xi)[t];
            const T au = sm.pml_at(xi, r, i);
            T ub = sm.row(D + xi)[t] + slot(res, xi * R + r, i, nx);
            T g = -dt * bb * au * ub;
            const T ubn = ub;
            ub = au * au * ub;
            if (final_) g += (T)0.5 * dt * bb * ub;
            P.u[xi][idx] = ub;
            slot(out, xi * R + r, i, nx) = g;
            if (P.hk_gb[0]) {
                const T gv = P.hk_gin[xi][idx];
                T add = ubn * (-dt * au * gv);
                if (final_) add += ub * (T)0.5 * dt * gv;
                P.hk_gb[xi][idx] += add;
            }
        }
    }
    __syncthreads();
    res = fft_rows<T, false>(out, res, P.fx, sm.tw, Q);
    r2c_unpack(res, P.spec, D, R, line0, nx, P.ldh);
}

// p_bar^n = -sum_xi D-_xi g_bar_xi (spectrum 0) + M^T h^n, then the tail.
template <typename T, int D>
__global__ void __launch_bounds__(256) k_adj_p(DevPlan<T> P, int R, int final_, const T* h_row, const T* qrow,
                                                T* gc2, const T* p0c) {
    RowSm<T, D> sm(P.nx, P.ldh, R);
    const int nx = P.nx, line0 = blockIdx.x * R;
    stage16(sm.tw, P.twx, (size_t)nx * sizeof(cplx<T>));
    adj_tail_prologue(sm, P, line0, final_);
    cp_commit();
    const int2 g = scatter_prologue(sm, P, line0, h_row);
    pdl_trigger();
    pdl_wait();
    stage_spectra(sm.S, P.spec, 1, line0, R, P.ldh);
    adj_tail_state(sm, P, line0, final_);
    cp_commit();
    cp_wait_all();
    __syncthreads();
    c2r_pack(sm.A, sm.S, 1, R, nx, P.ldh);
    __syncthreads();
    cplx<T>* res = fft_rows<T, true>(sm.A, sm.B, P.fx, sm.tw, R / 2);
    cplx<T>* other = (res == sm.A) ? sm.B : sm.A;
    scatter_rows(sm, P, g, res, line0, h_row);
    __syncthreads();
    adj_tail(sm, P, res, other, line0, final_, qrow, gc2, p0c);
}

// ------------------------------------------------------------------------------------------
// Spectral kernels: transforms along y (lax = 1) or z (lax = 2) of half-spectrum columns,
// with the k-space multiply fused in between for the multiply modes.
// blockIdx.x = tile of W columns kx; blockIdx.y = outer index (z for lax = 1, y for lax = 2).
//
// All fields a kernel transforms are interleaved in one tile [L][NF W] (field f, column c at
// f W + c), so one batched transform per direction covers them all.
// Shared memory: tw[L] | dpl[L] | dml[L] | cdp[8] | cdm[8] | X, Y, Z[L d W] (complex)
//                | kl2[Lpad] | ckx2[8] (real: squared wavenumbers)
// Symbols: kappa = sinc(c_ref |k| dt / 2) (k-space correction), |k|^(y-2), |k|^(y-1)
// (Eq. (state)), D+-_xi = i k_xi exp(+-i k_xi dx_xi / 2) (staggered grid); all scaled by 1/N.
// ------------------------------------------------------------------------------------------
// Multiplier of the first absorption channel: |k|^(y-2) / N (Eq. (state); zero at k = 0), or, in
// the time-reversal solve (tr_kc2 = 1 / k_c^2 > 0), -W(|k| / k_c) |k|^(y-2) / N with the radial
// Blackman window W(q) = 0.42 + 0.5 cos(pi q) + 0.08 cos(2 pi q) for q < 1 and 0 beyond (readings T1,
// T5: the absorption term reversed in sign and band-limited).
template <typename T> __device__ __forceinline__ T abs_mult0(const DevPlan<T>& P, T k2) {
    T s0 = (k2 > (T)0) ? pow(k2, P.pha) * P.invN : (T)0;
    if (P.tr_kc2 > (T)0) {
        const T q2 = k2 * P.tr_kc2;
        T w = 0;
        if (q2 < (T)1) {
            const T q = sqrt(q2);
            w = (T)0.42 + (T)0.5 * cospi(q) + (T)0.08 * cospi((T)2 * q);
        }
        s0 = -w * s0;
    }
    return s0;
}

template <typename T> size_t spec_smem_bytes(int D, int L, int W) {
    const int Lpad = (L + 3) & ~3;
    return (size_t)(3 * L + 16 + 3 * L * D * W) * sizeof(cplx<T>) + (size_t)(Lpad + 8) * sizeof(T);
}

// sinc(z) = sin(z)/z from its Taylor series in z^2 (alternating, terms z^2n / (2n+1)!), used for
// z^2 <= 4 where the truncation error is below the working precision; sin(z)/z otherwise.
template <typename T> __device__ __forceinline__ T sinc_sq(T z2);
template <> __device__ __forceinline__ float sinc_sq<float>(float z2) {
    if (z2 > 4.0f) {
        const float z = sqrtf(z2);
        return sinf(z) / z;
    }
    // 1/(2n+1)! for n = 0..9
    float r = 1.0f / 6402373705728000.0f;
    r = fmaf(r, -z2, 1.0f / 355687428096000.0f);
    r = fmaf(r, -z2, 1.0f / 1307674368000.0f);
    r = fmaf(r, -z2, 1.0f / 6227020800.0f);
    r = fmaf(r, -z2, 1.0f / 39916800.0f);
    r = fmaf(r, -z2, 1.0f / 362880.0f);
    r = fmaf(r, -z2, 1.0f / 5040.0f);
    r = fmaf(r, -z2, 1.0f / 120.0f);
    r = fmaf(r, -z2, 1.0f / 6.0f);
    return fmaf(r, -z2, 1.0f);
}
template <> __device__ __forceinline__ double sinc_sq<double>(double z2) {
    if (z2 > 4.0) {
        const double z = sqrt(z2);
        return sin(z) / z;
    }
    // 1/(2n+1)! for n = 0..12
    double r = 1.0 / 15511210043330985984000000.0;
    r = fma(r, -z2, 1.0 / 25852016738884976640000.0);
    r = fma(r, -z2, 1.0 / 51090942171709440000.0);
    r = fma(r, -z2, 1.0 / 121645100408832000.0);
    r = fma(r, -z2, 1.0 / 355687428096000.0);
    r = fma(r, -z2, 1.0 / 1307674368000.0);
    r = fma(r, -z2, 1.0 / 6227020800.0);
    r = fma(r, -z2, 1.0 / 39916800.0);
    r = fma(r, -z2, 1.0 / 362880.0);
    r = fma(r, -z2, 1.0 / 5040.0);
    r = fma(r, -z2, 1.0 / 120.0);
    r = fma(r, -z2, 1.0 / 6.0);
    return fma(r, -z2, 1.0);
}

template <typename T, int D, int MODE>
__global__ void __launch_bounds__(256) k_spec(DevPlan<T> P, int W, int lgW, int lax, int F) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int L = (lax == 1) ? P.ny : P.nz;
    const int Lpad = (L + 3) & ~3;
    cplx<T>* tw = reinterpret_cast<cplx<T>*>(smem_raw);
    cplx<T>* dpl = tw + L;
    cplx<T>* dml = dpl + L;
    cplx<T>* cdp = dml + L;
    cplx<T>* cdm = cdp + 8;
    cplx<T>* X = cdm + 8;
    const size_t TB = (size_t)L * D * W;   // one tile buffer
    cplx<T>* Y = X + TB;
    cplx<T>* Z = Y + TB;
    T* kl2 = reinterpret_cast<T*>(Z + TB);
    T* ckx2 = kl2 + Lpad;
    const FftAxis& ax = (lax == 1) ? P.fy : P.fz;
    const int kx0 = (blockIdx.x + P.tile0) * W;
    const int wv = min(W, P.nxh - kx0);
    const int outer = blockIdx.y;
    const size_t es = (lax == 1) ? (size_t)P.ldh : (size_t)P.ny * P.ldh;
    const size_t base = (lax == 1) ? (size_t)outer * P.ny * P.ldh + kx0 : (size_t)outer * P.ldh + kx0;
    constexpr bool MUL = (MODE != SPEC_PLAIN_FWD && MODE != SPEC_PLAIN_INV);
    // fields in and out of this kernel
    const int fin = (MODE == SPEC_GRAD) ? 1 : (MODE == SPEC_ABS ? 2 : (MUL ? D : F));
    const int fout = (MODE == SPEC_GRADT) ? 1 : (MODE == SPEC_ABS ? 2 : (MUL ? D : F));

    // ---- prologue: constant tables ----
    stage16(tw, (lax == 1) ? P.twy : P.twz, (size_t)L * sizeof(cplx<T>));
    T ko2 = 0;
    cplx<T> dpo = mkc<T>(0, 0), dmo = mkc<T>(0, 0);
    if constexpr (MUL) {
        const int la = (lax == 1) ? 1 : 2;
        stage16(dpl, P.dp[la], (size_t)L * sizeof(cplx<T>));
        stage16(dml, P.dm[la], (size_t)L * sizeof(cplx<T>));
        for (int i = threadIdx.x; i < L; i += blockDim.x) {
            const T k = P.kv[la][i];
            kl2[i] = k * k;
        }
        if (threadIdx.x < (unsigned)W) {
            const int kx = min(kx0 + (int)threadIdx.x, P.nxh - 1);
            cdp[threadIdx.x] = P.dp[0][kx];
            cdm[threadIdx.x] = P.dm[0][kx];
            const T k = P.kv[0][kx];
            ckx2[threadIdx.x] = k * k;
        }
        if (lax == 2) {
            const T ky = P.kv[1][outer];
            ko2 = ky * ky;
            dpo = P.dp[1][outer];
            dmo = P.dm[1][outer];
        }
    }
    cp_commit();
    pdl_trigger();
    pdl_wait();

    // ---- main load: every input field of the tile in flight at once ----
    const int LWin = fin * W;                                   // interleaved row length
    const int cb = ((size_t)W * sizeof(cplx<T>) >= 16) ? 16 : (int)sizeof(cplx<T>);   // chunk bytes
    const int epc = cb / (int)sizeof(cplx<T>);
    const int cpr = W / epc;                                     // chunks per field row
    for (int f = 0; f < fin; ++f) {
        const cplx<T>* src = P.spec[f] + base;
        for (int t = threadIdx.x; t < L * cpr; t += blockDim.x) {
            const int i = t / cpr, ch = t - i * cpr;
            cplx<T>* d = X + (size_t)i * LWin + f * W + ch * epc;
            const cplx<T>* g = src + (size_t)i * es + ch * epc;
            if (cb == 16) cp_async<16>(d, g);
            else cp_async<sizeof(cplx<T>)>(d, g);
        }
    }
    cp_commit();
    cp_wait_all();
    __syncthreads();

    // store field f of an interleaved tile with row length LW
    auto store = [&](const cplx<T>* buf, int LW, int f) {
        cplx<T>* dst = P.spec[f] + base;
        for (int t = threadIdx.x; t < L * W; t += blockDim.x) {
            const int i = t >> lgW, c = t & (W - 1);
            if (c < wv) dst[(size_t)i * es + c] = buf[(size_t)i * LW + f * W + c];
        }
    };
    auto lg = [](int v) { int l = 0; while ((1 << l) < v) ++l; return ((1 << l) == v) ? l : -1; };

    if constexpr (!MUL) {
        cplx<T>* r = (MODE == SPEC_PLAIN_FWD) ? fft_cols<T, false>(X, Y, ax, tw, LWin, lg(LWin))
                                              : fft_cols<T, true>(X, Y, ax, tw, LWin, lg(LWin));
        for (int f = 0; f < fout; ++f) store(r, LWin, f);
        return;
    } else {
        cplx<T>* res = fft_cols<T, false>(X, Y, ax, tw, LWin, lg(LWin));
        cplx<T>* spare = (res == X) ? Y : X;
        const int LWout = fout * W;
        // output tile: Z (GRAD: d fields from one input; GRADT: sum of d inputs; else in place)
        cplx<T>* O = (MODE == SPEC_GRAD || MODE == SPEC_GRADT) ? Z : res;
        for (int t = threadIdx.x; t < L * W; t += blockDim.x) {
            const int i = t >> lgW, c = t & (W - 1);
            const T k2 = ckx2[c] + kl2[i] + ko2;
            if constexpr (MODE == SPEC_ABS) {
                const T s0 = abs_mult0(P, k2);
                const T s1 = (k2 > (T)0) ? pow(k2, P.phb) * P.invN : (T)0;
                const size_t b0 = (size_t)i * LWin + c;
                O[b0] = cscale(res[b0], s0);
                O[b0 + W] = cscale(res[b0 + W], s1);
            } else {
                const T kap = sinc_sq(P.kap_a * P.kap_a * k2) * P.invN;
                constexpr bool plus = (MODE == SPEC_GRAD || MODE == SPEC_DIVT);
                const T sg = (MODE == SPEC_DIVT || MODE == SPEC_GRADT) ? -kap : kap;
                cplx<T> m[3];
                m[0] = plus ? cdp[c] : cdm[c];
                m[1] = (lax == 2) ? (plus ? dpo : dmo) : (plus ? dpl[i] : dml[i]);
                m[2] = plus ? dpl[i] : dml[i];
                if constexpr (MODE == SPEC_GRAD) {
                    const cplx<T> v = cscale(res[(size_t)i * W + c], sg);
#pragma unroll
                    for (int f = 0; f < D; ++f) O[(size_t)i * LWout + f * W + c] = cmul(v, m[f]);
                } else if constexpr (MODE == SPEC_GRADT) {
                    cplx<T> acc = mkc<T>(0, 0);
#pragma unroll
                    for (int f = 0; f < D; ++f) acc = cadd(acc, cmul(res[(size_t)i * LWin + f * W + c], m[f]));
                    O[(size_t)i * W + c] = cscale(acc, sg);
                } else {
#pragma unroll
                    for (int f = 0; f < D; ++f) {
                        const size_t b = (size_t)i * LWin + f * W + c;
                        O[b] = cscale(cmul(res[b], m[f]), sg);
                    }
                }
            }
        }
        __syncthreads();
        cplx<T>* r = fft_cols<T, true>(O, spare, ax, tw, LWout, lg(LWout));
        for (int f = 0; f < fout; ++f) store(r, LWout, f);
    }
}

}  // namespace pat
