// pat_persist.cuh -- the whole Nt-step solve of a 2-D grid as one persistent cooperative kernel.
//
// For grids whose state fits in the aggregate shared memory of the GPU (152 SMs x 227 KB), each
// CTA keeps the state and medium of its own x-lines resident in shared memory for all Nt steps:
// u_xi, rho_xi (or their adjoints), r / p_bar, c0^2, rho0, 1/rho0 on the staggered grids,
// c0^2 tau, c0^2 eta and the PML factors.  Per phase only the half spectra travel through L2:
//   row phase    x-transforms fused with the pointwise physics of the step (CTA b owns
//                x-line pairs [ppc b, ppc (b+1)));
//   column phase y-transforms with the k-space multiply (CTA b owns half-spectrum columns
//                [W b, W (b+1))).
// Phases are separated by a grid barrier whose wait is bounded: after ~2^25 polls the kernel
// records PAT_ETIMEOUT in the plan's status word and every CTA returns.  The arithmetic of every
// phase is the same as in the per-phase kernels of pat_kernels.cuh (Sec. II.A, Sec. III).
#pragma once

#include "pat_kernels.cuh"

namespace pat {

struct PersistCfg {
    int W, lgW;        // columns per CTA in column phases (power of two)
    int ntiles;        // ceil((nx/2 + 1) / W)
    int ppc;           // x-line pairs per CTA in row phases
    int rmax;          // 2 ppc
    int nres;          // resident real fields
};

constexpr unsigned long long kBarrierSpinLimit = 1ull << 25;

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier #k (k counted from 1) over `nblocks` CTAs: a monotonically increasing arrival
// counter (zeroed before the launch); barrier k completes when it reaches k * nblocks.
// Returns false (every thread of the CTA) if the wait ran out or another CTA reported an error.
__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}

// trace layout: [grid][nk][kTraceStride]: barrier entry, barrier exit, then sub-phase marks
constexpr int kTraceStride = 8;
struct TraceRef {
    unsigned long long* buf;
    int k0, nk;
};

// The wait is bounded twice: by `limit_ns` of %globaltimer (2 s by default) and by
// kBarrierSpinLimit polls; either way the CTA records PAT_ETIMEOUT and every CTA returns.
__device__ __forceinline__ bool grid_barrier(unsigned* gbar, unsigned nblocks, unsigned& k, int* abort_s,
                                             TraceRef tr = TraceRef{nullptr, 0, 0}, unsigned extra = 0,
                                             unsigned long long limit_ns = 2000000000ull) {
    __syncthreads();
    ++k;
    const int kt = (int)k - 1 - tr.k0;
    const bool traced = tr.buf && kt >= 0 && kt < tr.nk;
    if (threadIdx.x == 0) {
        if (traced) tr.buf[((size_t)blockIdx.x * tr.nk + kt) * kTraceStride] = globaltimer_ns();
        // arrival with release semantics at GPU scope: the CTA's writes (ordered before this by the
        // __syncthreads above) are visible to every CTA that observes the count; the polling load
        // has acquire semantics, and the __syncthreads below extends it to the whole CTA
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;\n" ::"l"(gbar) : "memory");
        const unsigned target = k * nblocks + extra;
        unsigned long long spins = 0;
        const unsigned long long t0 = globaltimer_ns();
        int ab = 0;
        // one load per poll: the error word of another CTA and the clock are looked at every 64th
        // poll, so the poll that sees the last arrival is not queued behind a second L2 round trip
        while (ld_acquire_gpu(&gbar[0]) < target) {
            if ((++spins & 63) != 0) continue;
            if (*(volatile unsigned*)&gbar[2] != 0u) {
                ab = 1;
                break;
            }
            if (spins > kBarrierSpinLimit || globaltimer_ns() - t0 > limit_ns) {
                atomicExch(&gbar[2], (unsigned)PAT_ETIMEOUT);
                ab = 1;
                break;
            }
        }
        if (traced) tr.buf[((size_t)blockIdx.x * tr.nk + kt) * kTraceStride + 1] = globaltimer_ns();
        *abort_s = ab;
    }
    __syncthreads();
    return *abort_s == 0;
}

template <typename T> struct PersistSm {
    cplx<T>* twx;
    cplx<T>* twy;
    cplx<T>* dpl;
    cplx<T>* dml;
    cplx<T>* cdp;
    cplx<T>* cdm;
    cplx<T>* work;   // row phase: A | B | S ; column phase: X | Y | Z
    cplx<T>* gb;     // power-of-two kernel: sensor gather / injection buffer (rows packed in pairs)
    T* res;          // resident fields [nres][rmax][nx]
    T* ax;           // a, au along x
    T* aux;
    T* ay;           // a, au of the CTA's lines (along y)
    T* auy;
    T* kl2;          // ky^2
    T* ckx2;         // kx^2 of the tile
    T* kapt;         // power-of-two kernel: kappa / N of the tile, [ky][c]
    T* s0t;          //   |k|^(y-2) / N and |k|^(y-1) / N of the tile (absorbing media)
    T* s1t;
    int* seg_i;
    T* seg_w;
    int* flag;
    int nx, rmax;
    TraceRef tr;
    const unsigned* kb;   // barriers passed so far
    __device__ T* row(int j) const { return res + j * rmax * nx; }
    // sub-phase mark j (call after a __syncthreads): time of the CTA reaching this point
    __device__ void mark(int j) const {
        if (!tr.buf || threadIdx.x != 0) return;
        const int kt = (int)*kb - tr.k0;
        if (kt >= 0 && kt < tr.nk) tr.buf[((size_t)blockIdx.x * tr.nk + kt) * kTraceStride + 2 + j] = globaltimer_ns();
    }
};

template <typename T> __host__ __device__ size_t persist_work_elems(int nx, int ny, int ldh, int rmax, int W) {
    const size_t rowp = (size_t)2 * rmax * nx + (size_t)2 * rmax * ldh;   // A, B (rmax lines) + S (2 fields)
    const size_t colp = (size_t)3 * ny * 2 * W;                           // X, Y, Z of [ny][2W]
    return rowp > colp ? rowp : colp;
}

template <typename T> size_t persist_smem_bytes(int nx, int ny, int ldh, int rmax, int W, int nres) {
    const int Lpad = (ny + 3) & ~3;
    size_t b = (size_t)(nx + 3 * ny + 16 + persist_work_elems<T>(nx, ny, ldh, rmax, W)) * sizeof(cplx<T>);
    b += (size_t)((size_t)nres * rmax * nx + 2 * nx + 2 * ((rmax + 3) & ~3) + Lpad + 8 + 2 * kSegCap) * sizeof(T);
    b += (size_t)(2 * kSegCap + 4) * sizeof(int);
    return b;
}

template <typename T> __device__ PersistSm<T> persist_carve(const DevPlan<T>& P, const PersistCfg& C) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PersistSm<T> s;
    s.nx = P.nx;
    s.rmax = C.rmax;
    s.twx = reinterpret_cast<cplx<T>*>(smem_raw);
    s.twy = s.twx + P.nx;
    s.dpl = s.twy + P.ny;
    s.dml = s.dpl + P.ny;
    s.cdp = s.dml + P.ny;
    s.cdm = s.cdp + 8;
    s.work = s.cdm + 8;
    s.res = reinterpret_cast<T*>(s.work + persist_work_elems<T>(P.nx, P.ny, P.ldh, C.rmax, C.W));
    s.ax = s.res + (size_t)C.nres * C.rmax * P.nx;
    s.aux = s.ax + P.nx;
    s.ay = s.aux + P.nx;
    s.auy = s.ay + ((C.rmax + 3) & ~3);
    s.kl2 = s.auy + ((C.rmax + 3) & ~3);
    s.ckx2 = s.kl2 + ((P.ny + 3) & ~3);
    s.seg_w = s.ckx2 + 8;
    s.seg_i = reinterpret_cast<int*>(s.seg_w + 2 * kSegCap);
    s.flag = s.seg_i + 2 * kSegCap;
    return s;
}

// ---- row-phase building blocks (lines line0 .. line0 + R - 1 of this CTA) ----
template <typename T>
__device__ cplx<T>* prow_c2r(const PersistSm<T>& s, const DevPlan<T>& P, int F, int line0, int R) {
    cplx<T>* A = s.work;
    cplx<T>* B = A + (size_t)s.rmax * P.nx;
    cplx<T>* S = B + (size_t)s.rmax * P.nx;
    stage_spectra(S, P.spec, F, line0, R, P.ldh);
    cp_commit();
    cp_wait_all();
    __syncthreads();
    s.mark(0);
    c2r_pack(A, S, F, R, P.nx, P.ldh);
    __syncthreads();
    s.mark(1);
    cplx<T>* r = fft_rows<T, true>(A, B, P.fx, s.twx, F * R / 2);
    s.mark(2);
    return r;
}
template <typename T> __device__ cplx<T>* prow_other(const PersistSm<T>& s, const DevPlan<T>& P, cplx<T>* res) {
    cplx<T>* A = s.work;
    return (res == A) ? A + (size_t)s.rmax * P.nx : A;
}
template <typename T>
__device__ void prow_r2c(const PersistSm<T>& s, const DevPlan<T>& P, cplx<T>* out, cplx<T>* scratch, int F,
                         int line0, int R) {
    __syncthreads();
    s.mark(3);
    cplx<T>* r = fft_rows<T, false>(out, scratch, P.fx, s.twx, F * R / 2);
    s.mark(4);
    r2c_unpack(r, P.spec, F, R, line0, P.nx, P.ldh);
    s.mark(5);
}

// sensor gather for the CTA's lines (pressure of line r = item r of buf)
template <typename T>
__device__ void pgather(const PersistSm<T>& s, const DevPlan<T>& P, int2 rng, int line0, const cplx<T>* buf,
                        T* data_row) {
    const DevSensors<T>& S = P.sens;
    const int nx = P.nx;
    for (int t = threadIdx.x; t < rng.y - rng.x; t += blockDim.x) {
        int j, pos;
        T w0, w1;
        if (t < kSegCap) {
            j = s.seg_i[2 * t];
            pos = s.seg_i[2 * t + 1];
            w0 = s.seg_w[2 * t];
            w1 = s.seg_w[2 * t + 1];
        } else {
            const int q = rng.x + t;
            j = S.g_seg_sensor[q];
            pos = (S.g_seg_line[q] - line0) * nx + S.g_seg_x0[q];
            w0 = S.g_seg_w0[q];
            w1 = S.g_seg_w1[q];
        }
        const int r = pos / nx, x = pos - r * nx;
        T acc = w0 * slot(buf, r, x, nx);
        if (w1 != (T)0) acc += w1 * slot(buf, r, x + 1, nx);
        atomicAdd(&data_row[j], acc);
    }
}

// adjoint injection p_bar += M^T h (segments = distinct points of the CTA's lines)
template <typename T>
__device__ void pscatter(const PersistSm<T>& s, const DevPlan<T>& P, int2 rng, int line0, cplx<T>* buf,
                         const T* h_row) {
    const DevSensors<T>& S = P.sens;
    const int nx = P.nx;
    for (int t = threadIdx.x; t < rng.y - rng.x; t += blockDim.x) {
        const int q = rng.x + t;
        T v = 0;
        for (int e = S.s_seg_e0[q]; e < S.s_seg_e0[q + 1]; ++e) v += S.s_ent_w[e] * h_row[S.s_ent_sensor[e]];
        const int pos = (t < kSegCap) ? s.seg_i[t] : (S.s_seg_line[q] - line0) * nx + S.s_seg_x[q];
        const int r = pos / nx, x = pos - r * nx;
        slot(buf, r, x, nx) += v;
    }
}

// ---- column phase: y-transform, multiply, inverse y-transform of the CTA's W columns ----
template <typename T, int MODE>
__device__ void pcol(const PersistSm<T>& s, const DevPlan<T>& P, int kx0, int W, int lgW) {
    constexpr int D = 2;
    const int L = P.ny;
    const size_t TB = (size_t)L * D * W;
    cplx<T>* X = s.work;
    cplx<T>* Y = X + TB;
    cplx<T>* Z = Y + TB;
    const int wv = min(W, P.nxh - kx0);
    const size_t es = (size_t)P.ldh;
    const size_t base = (size_t)kx0;
    const int fin = (MODE == SPEC_GRAD) ? 1 : 2;
    const int fout = (MODE == SPEC_GRADT) ? 1 : 2;
    const int LWin = fin * W, LWout = fout * W;
    if ((size_t)W * sizeof(cplx<T>) >= 16) {
        const int cpr = (int)((size_t)W * sizeof(cplx<T>) / 16);
        constexpr int EPC = 16 / (int)sizeof(cplx<T>);
        for (int f = 0; f < fin; ++f) {
            const cplx<T>* src = P.spec[f] + base;
            for (int t = threadIdx.x; t < L * cpr; t += blockDim.x) {
                const int i = t / cpr, ch = t - i * cpr;
                cp_async<16>(X + (size_t)i * LWin + f * W + ch * EPC, src + (size_t)i * es + ch * EPC);
            }
        }
        cp_commit();
        cp_wait_all();
    } else {
        // one complex float per row: 8-byte loads cached in L2 only (the spectra were written by
        // other CTAs in the previous phase), four in flight per thread
        for (int f = 0; f < fin; ++f) {
            const cplx<T>* src = P.spec[f] + base;
            for (int i0 = threadIdx.x; i0 < L; i0 += 4 * blockDim.x) {
                cplx<T> v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int i = i0 + u * blockDim.x;
                    if (i < L) v[u] = __ldcg(src + (size_t)i * es);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int i = i0 + u * blockDim.x;
                    if (i < L) X[(size_t)i * LWin + f * W] = v[u];
                }
            }
        }
    }
    __syncthreads();
    s.mark(0);
    auto lg = [](int v) { int l = 0; while ((1 << l) < v) ++l; return ((1 << l) == v) ? l : -1; };
    cplx<T>* res = fft_cols<T, false>(X, Y, P.fy, s.twy, LWin, lg(LWin));
    s.mark(1);
    cplx<T>* spare = (res == X) ? Y : X;
    cplx<T>* O = (MODE == SPEC_GRAD || MODE == SPEC_GRADT) ? Z : res;
    for (int t = threadIdx.x; t < L * W; t += blockDim.x) {
        const int i = t >> lgW, c = t & (W - 1);
        const T k2 = s.ckx2[c] + s.kl2[i];
        if constexpr (MODE == SPEC_ABS) {
            const T s0 = (k2 > (T)0) ? pow(k2, P.pha) * P.invN : (T)0;
            const T s1 = (k2 > (T)0) ? pow(k2, P.phb) * P.invN : (T)0;
            const size_t b0 = (size_t)i * LWin + c;
            O[b0] = cscale(res[b0], s0);
            O[b0 + W] = cscale(res[b0 + W], s1);
        } else {
            const T kap = sinc_sq(P.kap_a * P.kap_a * k2) * P.invN;
            constexpr bool plus = (MODE == SPEC_GRAD || MODE == SPEC_DIVT);
            const T sg = (MODE == SPEC_DIVT || MODE == SPEC_GRADT) ? -kap : kap;
            const cplx<T> m0 = plus ? s.cdp[c] : s.cdm[c];
            const cplx<T> m1 = plus ? s.dpl[i] : s.dml[i];
            if constexpr (MODE == SPEC_GRAD) {
                const cplx<T> v = cscale(res[(size_t)i * W + c], sg);
                O[(size_t)i * LWout + c] = cmul(v, m0);
                O[(size_t)i * LWout + W + c] = cmul(v, m1);
            } else if constexpr (MODE == SPEC_GRADT) {
                const cplx<T> acc = cadd(cmul(res[(size_t)i * LWin + c], m0), cmul(res[(size_t)i * LWin + W + c], m1));
                O[(size_t)i * W + c] = cscale(acc, sg);
            } else {
                const size_t b0 = (size_t)i * LWin + c;
                O[b0] = cscale(cmul(res[b0], m0), sg);
                O[b0 + W] = cscale(cmul(res[b0 + W], m1), sg);
            }
        }
    }
    __syncthreads();
    s.mark(2);
    cplx<T>* r = fft_cols<T, true>(O, spare, P.fy, s.twy, LWout, lg(LWout));
    s.mark(3);
    for (int f = 0; f < fout; ++f) {
        cplx<T>* dst = P.spec[f] + base;
        for (int t = threadIdx.x; t < L * W; t += blockDim.x) {
            const int i = t >> lgW, c = t & (W - 1);
            if (c < wv) dst[(size_t)i * es + c] = r[(size_t)i * LWout + f * W + c];
        }
    }
}

// resident field slots
enum PersistSlot : int { PS_U0 = 0, PS_U1, PS_R0, PS_R1, PS_RS, PS_C2, PS_RHO0, PS_B0, PS_B1, PS_C2TAU, PS_C2ETA };

template <typename T, bool ADJ>
__global__ void __launch_bounds__(256) k_persist(DevPlan<T> P, PersistCfg C, unsigned* gbar) {
    PersistSm<T> s = persist_carve<T>(P, C);
    const int nx = P.nx, ny = P.ny, b = blockIdx.x;
    const unsigned G = gridDim.x;
    const int pair0 = b * C.ppc;
    const int npair = max(0, min(ny / 2 - pair0, C.ppc));
    const int R = 2 * npair, line0 = 2 * pair0;
    const bool rows = R > 0, tile = b < C.ntiles;
    const int kx0 = b * C.W;
    const T dt = P.dt;
    const int Nt = P.Nt, Ns = P.sens.Ns;
    unsigned kbar = 0;
    const TraceRef TR{P.trace, P.trace_k0, P.trace_nk};
    s.tr = TR;
    s.kb = &kbar;

    // ---- setup: tables and resident medium ----
    stage16(s.twx, P.twx, (size_t)nx * sizeof(cplx<T>));
    stage16(s.twy, P.twy, (size_t)ny * sizeof(cplx<T>));
    stage16(s.dpl, P.dp[1], (size_t)ny * sizeof(cplx<T>));
    stage16(s.dml, P.dm[1], (size_t)ny * sizeof(cplx<T>));
    stage_elems(s.ax, P.a[0], nx);
    stage_elems(s.aux, P.au[0], nx);
    for (int i = threadIdx.x; i < ny; i += blockDim.x) {
        const T k = P.kv[1][i];
        s.kl2[i] = k * k;
    }
    if (threadIdx.x < (unsigned)C.W && tile) {
        const int kx = min(kx0 + (int)threadIdx.x, P.nxh - 1);
        s.cdp[threadIdx.x] = P.dp[0][kx];
        s.cdm[threadIdx.x] = P.dm[0][kx];
        const T k = P.kv[0][kx];
        s.ckx2[threadIdx.x] = k * k;
    }
    int2 seg = make_int2(0, 0);
    if (rows) {
        for (int r = threadIdx.x; r < R; r += blockDim.x) {
            s.ay[r] = P.a[1][line0 + r];
            s.auy[r] = P.au[1][line0 + r];
        }
        stage_rows(s.row(PS_C2), P.c2, line0, R, nx);
        stage_rows(s.row(PS_RHO0), P.rho0, line0, R, nx);
        stage_rows(s.row(PS_B0), P.b[0], line0, R, nx);
        stage_rows(s.row(PS_B1), P.b[1], line0, R, nx);
        if (P.lossy) {
            stage_rows(s.row(PS_C2TAU), P.c2tau, line0, R, nx);
            stage_rows(s.row(PS_C2ETA), P.c2eta, line0, R, nx);
        }
        if (!ADJ) stage_rows(s.row(PS_RS), P.img, line0, R, nx);   // p0 (consumed by the init)
        const DevSensors<T>& S = P.sens;
        if (!ADJ) {
            seg = make_int2(S.g_lineptr[line0], S.g_lineptr[line0 + R]);
            for (int t = threadIdx.x; t < min(seg.y - seg.x, kSegCap); t += blockDim.x) {
                const int q = seg.x + t;
                s.seg_i[2 * t] = S.g_seg_sensor[q];
                s.seg_i[2 * t + 1] = (S.g_seg_line[q] - line0) * nx + S.g_seg_x0[q];
                s.seg_w[2 * t] = S.g_seg_w0[q];
                s.seg_w[2 * t + 1] = S.g_seg_w1[q];
            }
        } else {
            seg = make_int2(S.s_lineptr[line0], S.s_lineptr[line0 + R]);
            for (int t = threadIdx.x; t < min(seg.y - seg.x, kSegCap); t += blockDim.x) {
                const int q = seg.x + t;
                s.seg_i[t] = (S.s_seg_line[q] - line0) * nx + S.s_seg_x[q];
            }
        }
    }
    cp_commit();
    cp_wait_all();
    __syncthreads();

    auto pml_a = [&](int xi, int r, int i) { return xi == 0 ? s.ax[i] : s.ay[r]; };
    auto pml_au = [&](int xi, int r, int i) { return xi == 0 ? s.aux[i] : s.auy[r]; };

    if constexpr (!ADJ) {
        // ================= forward: initial state, then Nt - 1 steps =================
        if (rows) {
            cplx<T>* A = s.work;
            for (int r = 0; r < R; ++r)
                for (int i = threadIdx.x; i < nx; i += blockDim.x) {
                    const int t = r * nx + i;
                    const T p = s.row(PS_RS)[t];
                    const T rh = p / ((T)2 * s.row(PS_C2)[t]);
                    s.row(PS_R0)[t] = rh;
                    s.row(PS_R1)[t] = rh;
                    slot(A, r, i, nx) = p;
                }
            __syncthreads();
            pgather(s, P, seg, line0, A, P.data);
            if (Nt > 1) prow_r2c(s, P, A, A + (size_t)s.rmax * nx, 1, line0, R);
        }
        if (Nt > 1 && !grid_barrier(gbar, G, kbar, s.flag, TR, P.bar_extra, P.bar_limit_ns)) return;
        for (int n = 0; n + 1 < Nt; ++n) {
            const bool last = (n + 2 == Nt);
            T* drow = P.data + (size_t)(n + 1) * Ns;
            // (1) g = D+ p
            if (tile) pcol<T, SPEC_GRAD>(s, P, kx0, C.W, C.lgW);
            if (!grid_barrier(gbar, G, kbar, s.flag, TR, P.bar_extra, P.bar_limit_ns)) return;
            // u update, x-FFT of u
            if (rows) {
                cplx<T>* res = prow_c2r(s, P, 2, line0, R);
                cplx<T>* out = prow_other(s, P, res);
                for (int r = 0; r < R; ++r)
                    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
                        const int t = r * nx + i;
#pragma unroll
                        for (int xi = 0; xi < 2; ++xi) {
                            const T g = slot(res, xi * R + r, i, nx);
                            const T bb = s.row(PS_B0 + xi)[t];
                            const T au = pml_au(xi, r, i);
                            const T uo = (n == 0) ? (T)0.5 * dt * bb * g : s.row(PS_U0 + xi)[t];
                            const T un = au * (au * uo - dt * bb * g);
                            s.row(PS_U0 + xi)[t] = un;
                            slot(out, xi * R + r, i, nx) = un;
                        }
                    }
                prow_r2c(s, P, out, res, 2, line0, R);
            }
            if (!grid_barrier(gbar, G, kbar, s.flag, TR, P.bar_extra, P.bar_limit_ns)) return;
            // (2) e = D- u
            if (tile) pcol<T, SPEC_DIV>(s, P, kx0, C.W, C.lgW);
            if (!grid_barrier(gbar, G, kbar, s.flag, TR, P.bar_extra, P.bar_limit_ns)) return;
            // rho update; lossless: p, sample; lossy: x-FFT of (dd, r)
            if (rows) {
                cplx<T>* res = prow_c2r(s, P, 2, line0, R);
                cplx<T>* out = prow_other(s, P, res);
                for (int r = 0; r < R; ++r)
                    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
                        const int t = r * nx + i;
                        const T rho0 = s.row(PS_RHO0)[t];
                        T rs = 0, es = 0;
#pragma unroll
                        for (int xi = 0; xi < 2; ++xi) {
                            const T e = slot(res, xi * R + r, i, nx);
                            const T a = pml_a(xi, r, i);
                            const T rh = a * (a * s.row(PS_R0 + xi)[t] - dt * rho0 * e);
                            s.row(PS_R0 + xi)[t] = rh;
                            rs += rh;
                            es += e;
                        }
                        if (P.lossy) {
                            s.row(PS_RS)[t] = rs;
                            slot(out, r, i, nx) = rho0 * es;
                            slot(out, R + r, i, nx) = rs;
                        } else {
                            slot(out, r, i, nx) = s.row(PS_C2)[t] * rs;
                        }
                    }
                if (!P.lossy) {
                    __syncthreads();
                    pgather(s, P, seg, line0, out, drow);
                    if (!last) prow_r2c(s, P, out, res, 1, line0, R);
                } else {
                    prow_r2c(s, P, out, res, 2, line0, R);
                }
            }
            if (P.lossy) {
                if (!grid_barrier(gbar, G, kbar, s.flag, TR, P.bar_extra, P.bar_limit_ns)) return;
                // (3) fractional Laplacians
                if (tile) pcol<T, SPEC_ABS>(s, P, kx0, C.W, C.lgW);
                if (!grid_barrier(gbar, G, kbar, s.flag, TR, P.bar_extra, P.bar_limit_ns)) return;
                if (rows) {
                    cplx<T>* res = prow_c2r(s, P, 2, line0, R);
                    cplx<T>* out = prow_other(s, P, res);
                    for (int r = 0; r < R; ++r)
                        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
                            const int t = r * nx + i;
                            const T Ld = slot(res, r, i, nx);
                            const T Lr = slot(res, R + r, i, nx);
                            slot(out, r, i, nx) = s.row(PS_C2)[t] * s.row(PS_RS)[t] + s.row(PS_C2TAU)[t] * Ld -
                                                  s.row(PS_C2ETA)[t] * Lr;
                        }
                    __syncthreads();
                    pgather(s, P, seg, line0, out, drow);
                    if (!last) prow_r2c(s, P, out, res, 1, line0, R);
                }
            }
            if (!last && !grid_barrier(gbar, G, kbar, s.flag, TR, P.bar_extra, P.bar_limit_ns)) return;
        }
    } else {
        // ================= adjoint: reverse time, exact transpose =================
        // resident: u_bar (PS_U0/1), rho_bar (PS_R0/1), p_bar (PS_RS)
        if (rows) {
            for (int j = 0; j < 4; ++j)
                for (int t = threadIdx.x; t < R * nx; t += blockDim.x) s.row(PS_U0 + j)[t] = 0;
        }
        // p_bar of time level n (items 0..R-1 of `pb`) -> final gradient, or the tail
        auto tail = [&](cplx<T>* pb, cplx<T>* other, bool final_) {
            if (final_) {
                for (int r = 0; r < R; ++r)
                    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
                        const int t = r * nx + i;
                        const T sr = s.row(PS_R0)[t] + s.row(PS_R1)[t];
                        P.img[(size_t)(line0 + r) * nx + i] = slot(pb, r, i, nx) + sr / ((T)2 * s.row(PS_C2)[t]);
                    }
                return;
            }
            for (int r = 0; r < R; ++r)
                for (int i = threadIdx.x; i < nx; i += blockDim.x) {
                    const int t = r * nx + i;
                    const T pv = slot(pb, r, i, nx);
                    if (P.lossy) {
                        s.row(PS_RS)[t] = pv;
                        slot(other, r, i, nx) = s.row(PS_C2TAU)[t] * pv;
                        slot(other, R + r, i, nx) = s.row(PS_C2ETA)[t] * pv;
                    } else {
                        const T rbar = s.row(PS_C2)[t] * pv;
                        const T rho0 = s.row(PS_RHO0)[t];
#pragma unroll
                        for (int xi = 0; xi < 2; ++xi) {
                            const T a = pml_a(xi, r, i);
                            const T rb = s.row(PS_R0 + xi)[t] + rbar;
                            slot(other, xi * R + r, i, nx) = -dt * rho0 * a * rb;
                            s.row(PS_R0 + xi)[t] = a * a * rb;
                        }
                    }
                }
            prow_r2c(s, P, other, pb, 2, line0, R);
        };
        if (rows) {
            cplx<T>* A = s.work;
            cplx<T>* B = A + (size_t)s.rmax * nx;
            for (int r = 0; r < R; ++r)
                for (int i = threadIdx.x; i < nx; i += blockDim.x) slot(A, r, i, nx) = 0;
            __syncthreads();
            pscatter(s, P, seg, line0, A, P.data + (size_t)(Nt - 1) * Ns);
            __syncthreads();
            tail(A, B, Nt == 1);
        }
        if (Nt == 1) return;
        if (!grid_barrier(gbar, G, kbar, s.flag, TR, P.bar_extra, P.bar_limit_ns)) return;
        for (int n = Nt - 2; n >= 0; --n) {
            const bool final_ = (n == 0);
            if (P.lossy) {
                if (tile) pcol<T, SPEC_ABS>(s, P, kx0, C.W, C.lgW);
                if (!grid_barrier(gbar, G, kbar, s.flag, TR, P.bar_extra, P.bar_limit_ns)) return;
                if (rows) {
                    cplx<T>* res = prow_c2r(s, P, 2, line0, R);
                    cplx<T>* out = prow_other(s, P, res);
                    for (int r = 0; r < R; ++r)
                        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
                            const int t = r * nx + i;
                            const T ddbar = slot(res, r, i, nx);
                            const T w = slot(res, R + r, i, nx);
                            const T rbar = s.row(PS_C2)[t] * s.row(PS_RS)[t] - w;
                            const T rho0 = s.row(PS_RHO0)[t];
#pragma unroll
                            for (int xi = 0; xi < 2; ++xi) {
                                const T a = pml_a(xi, r, i);
                                const T rb = s.row(PS_R0 + xi)[t] + rbar;
                                slot(out, xi * R + r, i, nx) = rho0 * ddbar - dt * rho0 * a * rb;
                                s.row(PS_R0 + xi)[t] = a * a * rb;
                            }
                        }
                    prow_r2c(s, P, out, res, 2, line0, R);
                }
                if (!grid_barrier(gbar, G, kbar, s.flag, TR, P.bar_extra, P.bar_limit_ns)) return;
            }
            // transpose of e = D- u
            if (tile) pcol<T, SPEC_DIVT>(s, P, kx0, C.W, C.lgW);
            if (!grid_barrier(gbar, G, kbar, s.flag, TR, P.bar_extra, P.bar_limit_ns)) return;
            if (rows) {
                cplx<T>* res = prow_c2r(s, P, 2, line0, R);
                cplx<T>* out = prow_other(s, P, res);
                for (int r = 0; r < R; ++r)
                    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
                        const int t = r * nx + i;
#pragma unroll
                        for (int xi = 0; xi < 2; ++xi) {
                            const T bb = s.row(PS_B0 + xi)[t];
                            const T au = pml_au(xi, r, i);
                            T ub = s.row(PS_U0 + xi)[t] + slot(res, xi * R + r, i, nx);
                            T g = -dt * bb * au * ub;
                            ub = au * au * ub;
                            if (final_) g += (T)0.5 * dt * bb * ub;
                            s.row(PS_U0 + xi)[t] = ub;
                            slot(out, xi * R + r, i, nx) = g;
                        }
                    }
                prow_r2c(s, P, out, res, 2, line0, R);
            }
            if (!grid_barrier(gbar, G, kbar, s.flag, TR, P.bar_extra, P.bar_limit_ns)) return;
            // transpose of g = D+ p
            if (tile) pcol<T, SPEC_GRADT>(s, P, kx0, C.W, C.lgW);
            if (!grid_barrier(gbar, G, kbar, s.flag, TR, P.bar_extra, P.bar_limit_ns)) return;
            if (rows) {
                cplx<T>* res = prow_c2r(s, P, 1, line0, R);
                cplx<T>* other = prow_other(s, P, res);
                pscatter(s, P, seg, line0, res, P.data + (size_t)n * Ns);
                __syncthreads();
                tail(res, other, final_);
            }
            if (!final_ && !grid_barrier(gbar, G, kbar, s.flag, TR, P.bar_extra, P.bar_limit_ns)) return;
        }
    }
}

}  // namespace pat
