// pat_persist2.cuh -- the persistent 2-D solve for power-of-two grids, with register-fused
// transforms.
//
// Same resident-state scheme, phases, barriers and arithmetic as k_persist (pat_persist.cuh);
// what changes is how a phase moves its data.  The generic phase stages the half spectra in
// shared memory, packs them, runs an inverse transform (one shared-memory round trip per stage),
// applies the physics, runs the forward transform and unpacks: ten shared-memory passes and nine
// CTA barriers.  Here, for n = 2^lg, the Stockham schedule is fixed -- forward radices
// (r0, 8, ..., 8), inverse radices the reverse (8, ..., 8, r0) -- so that
//   * the first stage of a transform loads its operands straight from the L2-resident spectra
//     (the C2R packing of two real lines is done on the loaded values);
//   * the last stage of the first transform and the first stage of the second one act on the
//     same elements {j + r n / R}: the thread that finishes butterfly j keeps its outputs in
//     registers, applies the pointwise physics (row phase) or the k-space multiply (column phase)
//     and runs the next transform's first butterfly on them;
//   * the last forward x-stage holds both X[k] and X[n - k] in one thread (it takes butterflies j
//     and m - j), so the R2C unpacking and the store to the spectra happen in registers.
// A phase is then four shared-memory round trips for n = 512 and two for n = 64.  Shared-memory
// lines are XOR-swizzled (element e at e ^ ((e >> 3) & 15)) so that the strided Stockham stores
// are free of bank conflicts, and every stage reads its twiddles from its own table laid out
// [r - 1][k], consecutive in k.
#pragma once

#include <type_traits>

#include "pat_persist.cuh"
#include "pat_p2.h"

namespace pat {

__device__ __forceinline__ int swz(int e) { return e ^ ((e >> 3) & 15); }
// Start of line q in a line buffer whose fields hold 2^lgnl lines each.  Fields sit 64 bytes
// beyond whole lines (p2_field_pad), so that the lane pairs of the fused stages, which touch the
// same element of two fields, hit different banks.
// lp > 0 adds lp elements after every line as well (kernels whose lanes step across lines).
// (shared-memory offsets: 32-bit)
template <typename T> __device__ __forceinline__ int lbase(int q, int n, int lgnl, int lp = 0) {
    return q * (n + lp) + (q >> lgnl) * p2_field_pad<T>();
}
template <int R> struct Lg2 { static constexpr int v = R == 2 ? 1 : (R == 4 ? 2 : (R == 8 ? 3 : 4)); };

// The swizzle is linear over XOR: swz(a ^ b) = swz(a) ^ swz(b).  Element j + r m of a butterfly
// (j < m, m a power of two) is j ^ (r m), and an output b + r Ns of a Stockham store is b ^ (r Ns)
// (disjoint bits), so their swizzled indices are the thread's swz(j) or swz(b) XOR a per-r term.
// With the line length fixed at compile time (CM) that term is a constant; when r m is a multiple
// of 16 it splits into a XOR of the low four bits and an added offset (swz(j) has no bit of r m),
// which the loads take as an immediate.
__device__ __forceinline__ int swz_xor(int sj, int rm) {
    return (rm % 16 == 0) ? (sj ^ ((rm >> 3) & 15)) + rm : sj ^ swz(rm);
}

// butterfly j of a stage (span Ns, stride m = n / R): load elements j + r m of `src`, twiddle
template <typename T, int R, bool INV, bool CM = false>
__device__ __forceinline__ void p2_load(cplx<T> (&v)[R], const cplx<T>* src, int j, int m, int Ns,
                                        const cplx<T>* tws) {
    if constexpr (CM) {
        const int sj = swz(j);
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src[swz_xor(sj, r * m)];
    } else {
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src[swz(j + r * m)];
    }
    if (Ns > 1) {
        const int k = j & (Ns - 1);
#pragma unroll
        for (int r = 1; r < R; ++r) {
            const cplx<T> w = tws[(r - 1) * Ns + k];
            v[r] = INV ? cmulc(v[r], w) : cmul(v[r], w);
        }
    }
}
template <typename T, int R, bool CM = false>
__device__ __forceinline__ void p2_store(cplx<T>* dst, int j, int Ns, const cplx<T> (&v)[R]) {
    const int k = j & (Ns - 1);
    const int b = (j - k) * R + k;
    if constexpr (CM) {
        // Ns >= 16: bits 0..3 of b are those of k, so swz(b) leaves the bits of r Ns clear
        const int sb = swz(b);
#pragma unroll
        for (int r = 0; r < R; ++r)
            dst[Ns % 16 == 0 ? (sb ^ ((r * Ns >> 3) & 15)) + r * Ns : sb ^ swz(r * Ns)] = v[r];
    } else {
#pragma unroll
        for (int r = 0; r < R; ++r) dst[swz(b + r * Ns)] = v[r];
    }
}

// the middle stages 1 .. nst-2 (radix 8) over `nlines` lines, each followed by a CTA barrier
template <typename T, bool INV, class AX>
__device__ cplx<T>* p2_mid(cplx<T>* a, cplx<T>* b, const AX& ax, const cplx<T>* tab, int nlines, int lgnl,
                          int lp = 0) {
    constexpr bool CM = P2IsC<AX>::value;
    const int lgm = ax.lg - 3, m = 1 << lgm;
#pragma unroll
    for (int s = 1; s + 1 < ax.nst; ++s) {
        const int Ns = INV ? p2_ins(s) : p2_fns(ax, s);
        const cplx<T>* tws = tab + (INV ? p2_off_i(ax, s) : p2_off_f(ax, s));
        for (int t = threadIdx.x; t < (nlines << lgm); t += blockDim.x) {
            const int line = t >> lgm, j = t & (m - 1);
            cplx<T> v[8];
            p2_load<T, 8, INV, CM>(v, a + lbase<T>(line, ax.n, lgnl, lp), j, m, Ns, tws);
            dft<T, 8, INV>(v);
            p2_store<T, 8, CM>(b + lbase<T>(line, ax.n, lgnl, lp), j, Ns, v);
        }
        __syncthreads();
        cplx<T>* tmp = a;
        a = b;
        b = tmp;
    }
    return a;
}

template <class Fn> __device__ __forceinline__ void with_radix(int r, Fn&& fn) {
    if (r == 8) fn(std::integral_constant<int, 8>{});
    else if (r == 4) fn(std::integral_constant<int, 4>{});
    else fn(std::integral_constant<int, 2>{});
}

// ---------------------------------------------------------------------------------------------
// row phase: complex line q = f np + p holds rows 2p (real part) and 2p + 1 (imaginary part) of
// field f of the CTA's R = 2 np rows
// ---------------------------------------------------------------------------------------------
// Stage the half spectra of FI fields for the CTA's R rows (one contiguous block per field) into
// S (row q of field f at S + (f R + q) ldh); asynchronous, completed by the caller's wait.
template <typename T>
__device__ __forceinline__ void p2_row_stage(cplx<T>* S, cplx<T>* const* spec, int FI, int R, int line0, int ldh) {
    for (int f = 0; f < FI; ++f)
        stage16(S + (size_t)f * R * ldh, spec[f] + (size_t)line0 * ldh, (size_t)R * ldh * sizeof(cplx<T>));
    cp_commit();
}

// inverse x-stage 0 (radix 8, no twiddles) on the C2R packing of the staged half spectra
template <typename T, class AX>
__device__ void p2_row_in(cplx<T>* dst, const cplx<T>* S, int FI, int np, int lgnp, const AX& ax, int ldh) {
    const int n = ax.n, lgm = ax.lg - 3, m = 1 << lgm, half = n >> 1;
    for (int t = threadIdx.x; t < ((FI * np) << lgm); t += blockDim.x) {
        const int q = t >> lgm, j = t & (m - 1);
        const int f = q / np, p = q - f * np;
        const cplx<T>* a = S + (f * 2 * np + 2 * p) * ldh;
        const cplx<T>* b = a + ldh;
        cplx<T> A[8], B[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int k = j + r * m;
            const int kk = k <= half ? k : n - k;
            A[r] = a[kk];
            B[r] = b[kk];
        }
        cplx<T> v[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int k = j + r * m;
            if (k == 0 || k == half) {
                A[r].y = 0;
                B[r].y = 0;
            }
            v[r] = (k <= half) ? mkc<T>(A[r].x - B[r].y, A[r].y + B[r].x)    // A + i B
                               : mkc<T>(A[r].x + B[r].y, B[r].x - A[r].y);   // conj(A) + i conj(B)
        }
        dft<T, 8, true>(v);
        p2_store<T, 8, P2IsC<AX>::value>(dst + lbase<T>(q, n, lgnp), j, 1, v);
    }
}

template <typename T> __device__ __forceinline__ cplx<T> shfl_pair(cplx<T> v) {
    v.x = __shfl_xor_sync(0xffffffffu, v.x, 1);
    v.y = __shfl_xor_sync(0xffffffffu, v.y, 1);
    return v;
}

// Element loop of the pointwise step of a fused row stage: f(row, x, in[FI], out[FO]) for the
// 2 H real elements this thread owns (positions r = h H + k of butterfly j; rows 2p, 2p + 1;
// x = j + r m)
template <typename T, int H, int FI, int FO, class F>
__device__ __forceinline__ void p2_each(int p, int j, int m, int h, const cplx<T> (&z)[2][H], cplx<T> (&o)[2][H],
                                        F&& f) {
#pragma unroll
    for (int k = 0; k < H; ++k) {
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            T in[2], out[2] = {};
#pragma unroll
            for (int q = 0; q < FI; ++q) in[q] = hh ? z[q][k].y : z[q][k].x;
            f(2 * p + hh, j + (h * H + k) * m, in, out);
#pragma unroll
            for (int g = 0; g < FO; ++g) {
                if (hh) o[g][k].y = out[g];
                else o[g][k].x = out[g];
            }
        }
    }
}

// Last inverse x-stage (radix R, Ns = n / R), the pointwise step, and -- when `fwd` -- forward
// x-stage 0, run by lane pairs (2u, 2u + 1) on butterfly u = (p, j).  Lane h transforms input
// field h (both lanes field 0 when FI = 1); one exchange gives each lane every field at its half
// of the positions (r = h H + k), where it runs pw(p, j, m, h, zi, oo); a second exchange gives
// lane h every position of output field h, which it transforms and stores (FO = 1: both lanes
// transform field 0 and each stores its half).  FI = 0: pw reads its inputs itself.
template <typename T, int R, class AX, class PW>
__device__ __forceinline__ void p2_row_fuse(const cplx<T>* src, cplx<T>* dst, const cplx<T>* tab, const AX& ax,
                                            int np, int lgnp, int FI, int FO, bool fwd, PW&& pw) {
    constexpr int H = R / 2;
    constexpr bool CM = P2IsC<AX>::value;
    const int n = ax.n, lgm = ax.lg - Lg2<R>::v, m = 1 << lgm;
    const cplx<T>* twl = tab + p2_off_i(ax, ax.nst - 1);
    const int total = (np << lgm) * 2;
    for (int t0 = 0; t0 < total; t0 += blockDim.x) {   // uniform trip count: whole warps shuffle
        const int t = t0 + (int)threadIdx.x;
        const bool valid = t < total;
        const int h = t & 1, u = t >> 1;
        const int p = u >> lgm, j = u & (m - 1);
        cplx<T> z[R];
        if (valid && FI > 0) {
            p2_load<T, R, true, CM>(z, src + lbase<T>((FI == 2 ? h : 0) * np + p, n, lgnp), j, m, m, twl);
            dft<T, R, true>(z);
        }
        cplx<T> zi[2][H], oo[2][H];
#pragma unroll
        for (int k = 0; k < H; ++k) {
            const cplx<T> mine = h ? z[H + k] : z[k];
            zi[0][k] = mine;
            if (FI == 2) {
                const cplx<T> recv = shfl_pair<T>(h ? z[k] : z[H + k]);
                zi[0][k] = h ? recv : mine;
                zi[1][k] = h ? mine : recv;
            }
        }
        if (valid) pw(p, j, m, h, zi, oo);
        if (!fwd) continue;
        cplx<T> w[R];
#pragma unroll
        for (int k = 0; k < H; ++k) {
            const cplx<T> own = (FO == 2 && h) ? oo[1][k] : oo[0][k];
            const cplx<T> rcv = shfl_pair<T>((FO == 2 && !h) ? oo[1][k] : oo[0][k]);
            w[k] = h ? rcv : own;
            w[H + k] = h ? own : rcv;
        }
        if (!valid) continue;
        dft<T, R, false>(w);
        cplx<T>* d = dst + lbase<T>((FO == 2 ? h : 0) * np + p, n, lgnp);
        if (FO == 2) {
            p2_store<T, R, CM>(d, j, 1, w);
        } else {
#pragma unroll
            for (int k = 0; k < H; ++k) d[swz(j * R + h * H + k)] = h ? w[H + k] : w[k];
        }
    }
}

// last forward x-stage (radix 8, Ns = n / 8) and R2C unpacking into the half spectra: unit u of a
// line runs butterflies u and m - u (u = 0: 0 and m / 2), which hold every X[k] with its X[n - k]
template <typename T, class AX>
__device__ void p2_row_out(const cplx<T>* src, cplx<T>* const* spec, const cplx<T>* tab, const AX& ax,
                           int FO, int np, int lgnp, int line0, int ldh) {
    constexpr bool CM = P2IsC<AX>::value;
    const int n = ax.n, lgm = ax.lg - 3, m = 1 << lgm, lgh = lgm - 1, hm = m >> 1;
    const cplx<T>* twl = tab + p2_off_f(ax, ax.nst - 1);
    for (int t = threadIdx.x; t < ((FO * np) << lgh); t += blockDim.x) {
        const int q = t >> lgh, u = t & (hm - 1);
        const int f = q / np, p = q - f * np;
        const int j1 = u, j2 = (u == 0) ? hm : m - u;
        const cplx<T>* line = src + lbase<T>(q, n, lgnp);
        cplx<T> X1[8], X2[8];
        p2_load<T, 8, false, CM>(X1, line, j1, m, m, twl);
        p2_load<T, 8, false, CM>(X2, line, j2, m, m, twl);
        dft<T, 8, false>(X1);
        dft<T, 8, false>(X2);
        cplx<T>* a = spec[f] + (size_t)(line0 + 2 * p) * ldh;
        cplx<T>* b = a + ldh;
        auto put = [&](int k, cplx<T> zk, cplx<T> zm) {
            a[k] = mkc<T>((T)0.5 * (zk.x + zm.x), (T)0.5 * (zk.y - zm.y));
            b[k] = mkc<T>((T)0.5 * (zk.y + zm.y), (T)0.5 * (zm.x - zk.x));
        };
        if (u != 0) {
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                put(j1 + r * m, X1[r], X2[7 - r]);
                put(j2 + r * m, X2[r], X1[7 - r]);
            }
        } else {
#pragma unroll
            for (int r = 0; r <= 4; ++r) put(r * m, X1[r], X1[(8 - r) & 7]);
#pragma unroll
            for (int r = 0; r < 4; ++r) put(hm + r * m, X2[r], X2[7 - r]);
        }
    }
}

// ---------------------------------------------------------------------------------------------
// column phase: line q = f W + c is column kx0 + c of field f (length ny)
// ---------------------------------------------------------------------------------------------
// Stage columns [kx0, kx0 + W) of FI fields into S ([f][ky][c]).  Tiles reach into the zeroed
// padding columns of the half spectra (kx0 + W <= ldh).  Pieces of 16 bytes go through cp.async
// (L2 only); narrower ones are loaded with ld.global.cg (L1 is not coherent with the other CTAs'
// writes of the previous phase) and stored synchronously.
template <typename T>
__device__ __forceinline__ void p2_col_stage(cplx<T>* S, cplx<T>* const* spec, int FI, int W, int kx0, int ny,
                                             int ldh) {
    const int cb = W * (int)sizeof(cplx<T>);
    if (cb >= 16) {
        const int cpr = cb / 16;
        constexpr int EPC = 16 / (int)sizeof(cplx<T>);
        for (int f = 0; f < FI; ++f) {
            const cplx<T>* src = spec[f] + kx0;
            cplx<T>* d = S + f * ny * W;
            for (int t = threadIdx.x; t < ny * cpr; t += blockDim.x) {
                const int i = t / cpr, ch = t - i * cpr;
                cp_async<16>(d + i * W + ch * EPC, src + (size_t)i * ldh + ch * EPC);
            }
        }
        cp_commit();
    } else {
        for (int f = 0; f < FI; ++f) {
            const cplx<T>* src = spec[f] + kx0;
            cplx<T>* d = S + (size_t)f * ny;
            for (int i0 = threadIdx.x; i0 < ny; i0 += 4 * blockDim.x) {
                cplx<T> v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int i = i0 + u * blockDim.x;
                    if (i < ny) v[u] = __ldcg(src + (size_t)i * ldh);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int i = i0 + u * blockDim.x;
                    if (i < ny) d[i] = v[u];
                }
            }
        }
    }
}

// forward y-stage 0 (radix R, no twiddles) on the staged columns
template <typename T, int R, class AX>
__device__ void p2_col_in(cplx<T>* dst, const cplx<T>* S, int FI, int W, int lgW, const AX& ay) {
    const int n = ay.n, lgm = ay.lg - Lg2<R>::v, m = 1 << lgm;
    for (int t = threadIdx.x; t < ((FI * W) << lgm); t += blockDim.x) {
        const int c = t & (W - 1), j = (t >> lgW) & (m - 1), f = t >> (lgW + lgm);
        const cplx<T>* src = S + (f * n + j) * W + c;   // staged columns [f][ky][c], ky = j + r m
        const int step = m * W;
        cplx<T> v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src[r * step];
        dft<T, R, false>(v);
        p2_store<T, R, P2IsC<AX>::value>(dst + lbase<T>(f * W + c, n, lgW), j, 1, v);
    }
}

// last forward y-stage (radix 8, Ns = n / 8), the k-space multiply of `mode`, inverse y-stage 0,
// by lane pairs (2u, 2u + 1) on butterfly u = (c, j): lane h transforms field h (both lanes field 0
// when one field comes in) and produces output field h (both lanes the single output of GRADT,
// each storing half).  The multipliers of the CTA's tile are resident: kapt = kappa / N, s0t /
// s1t = |k|^(y-2) / N and |k|^(y-1) / N (Eq. Twelve's fractional Laplacians), [ky][c]; the shift
// operators per column (cdp / cdm) and per row (dpl / dml).
template <typename T, class AX>
__device__ __forceinline__ void p2_col_fuse(const PersistSm<T>& s, const cplx<T>* src, cplx<T>* dst,
                                            const AX& ay, int W, int lgW, int mode) {
    constexpr bool CM = P2IsC<AX>::value;
    const int fi = (mode == SPEC_GRAD) ? 1 : 2, fo = (mode == SPEC_GRADT) ? 1 : 2;
    const int n = ay.n, lgm = ay.lg - 3, m = 1 << lgm;
    const cplx<T>* twl = s.twy + p2_off_f(ay, ay.nst - 1);
    const int total = (W << lgm) * 2;
    for (int t0 = 0; t0 < total; t0 += blockDim.x) {   // uniform trip count: whole warps shuffle
        const int t = t0 + (int)threadIdx.x;
        const bool valid = t < total;
        const int h = t & 1, u = t >> 1;
        const int c = u & (W - 1), j = u >> lgW;
        cplx<T> z[8], o[8];
        if (valid) {
            p2_load<T, 8, false, CM>(z, src + lbase<T>((fi == 2 ? h : 0) * W + c, n, lgW), j, m, m, twl);
            dft<T, 8, false>(z);
        }
        switch (mode) {
            case SPEC_ABS: {
                const T* sf = h ? s.s1t : s.s0t;
#pragma unroll
                for (int r = 0; r < 8; ++r) o[r] = cscale(z[r], valid ? sf[(j + r * m) * W + c] : (T)0);
            } break;
            case SPEC_GRAD: {
                const cplx<T> m0 = s.cdp[c];
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    const int i = valid ? j + r * m : 0;
                    const cplx<T> v = cscale(z[r], s.kapt[i * W + c]);
                    o[r] = cmul(v, h ? s.dpl[i] : m0);
                }
            } break;
            case SPEC_GRADT: {
                const cplx<T> m0 = s.cdm[c];
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    const int i = valid ? j + r * m : 0;
                    const cplx<T> mine = cmul(z[r], h ? s.dml[i] : m0);
                    const cplx<T> other = shfl_pair<T>(mine);
                    o[r] = cscale(h ? cadd(other, mine) : cadd(mine, other), -s.kapt[i * W + c]);
                }
            } break;
            case SPEC_DIV: {
                const cplx<T> m0 = s.cdm[c];
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    const int i = valid ? j + r * m : 0;
                    o[r] = cscale(cmul(z[r], h ? s.dml[i] : m0), s.kapt[i * W + c]);
                }
            } break;
            default: {   // SPEC_DIVT
                const cplx<T> m0 = s.cdp[c];
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    const int i = valid ? j + r * m : 0;
                    o[r] = cscale(cmul(z[r], h ? s.dpl[i] : m0), -s.kapt[i * W + c]);
                }
            } break;
        }
        if (!valid) continue;
        dft<T, 8, true>(o);
        cplx<T>* d = dst + lbase<T>((fo == 2 ? h : 0) * W + c, n, lgW);
        if (fo == 2) {
            p2_store<T, 8, CM>(d, j, 1, o);
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) d[swz(j * 8 + h * 4 + k)] = h ? o[4 + k] : o[k];
        }
    }
}

// last inverse y-stage (radix R, Ns = n / R), stored to the spectra (valid columns only)
template <typename T, int R, class AX>
__device__ void p2_col_out(const cplx<T>* src, cplx<T>* const* spec, const cplx<T>* tab, int FO, int W, int lgW,
                           int kx0, int wv, const AX& ay, int ldh) {
    const int n = ay.n, lgm = ay.lg - Lg2<R>::v, m = 1 << lgm;
    const cplx<T>* twl = tab + p2_off_i(ay, ay.nst - 1);
    for (int t = threadIdx.x; t < ((FO * W) << lgm); t += blockDim.x) {
        const int c = t & (W - 1), j = (t >> lgW) & (m - 1), f = t >> (lgW + lgm);
        cplx<T> v[R];
        p2_load<T, R, true, P2IsC<AX>::value>(v, src + lbase<T>(f * W + c, n, lgW), j, m, m, twl);
        dft<T, R, true>(v);
        if (c < wv) {
            cplx<T>* dst = spec[f] + kx0 + c + (size_t)j * ldh;
            const size_t mld = (size_t)m * ldh;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                *dst = v[r];
                dst += mld;
            }
        }
    }
}

// whole column phase of `mode` for columns [kx0, kx0 + W)
template <typename T, class AX>
__device__ __forceinline__ void p2_col(const PersistSm<T>& s, const DevPlan<T>& P, const AX& ay, int kx0, int W,
                                       int lgW, int mode) {
    const int fi = (mode == SPEC_GRAD) ? 1 : 2, fo = (mode == SPEC_GRADT) ? 1 : 2;
    cplx<T>* A = s.work;
    cplx<T>* B = A + (size_t)2 * W * ay.n + p2_field_pad<T>();
    p2_col_stage<T>(B, P.spec, fi, W, kx0, ay.n, P.ldh);
    cp_wait_all();
    __syncthreads();
    s.mark(0);
    with_radix(ay.r0, [&](auto RC) { p2_col_in<T, decltype(RC)::value>(A, B, fi, W, lgW, ay); });
    __syncthreads();
    s.mark(1);
    cplx<T>* a = p2_mid<T, false>(A, B, ay, s.twy, fi * W, lgW);
    cplx<T>* b = (a == A) ? B : A;
    s.mark(2);
    p2_col_fuse<T>(s, a, b, ay, W, lgW, mode);
    __syncthreads();
    s.mark(3);
    a = p2_mid<T, true>(b, a, ay, s.twy, fo * W, lgW);
    s.mark(4);
    const int wv = min(W, P.nxh - kx0);
    with_radix(ay.r0, [&](auto RC) {
        p2_col_out<T, decltype(RC)::value>(a, P.spec, s.twy, fo, W, lgW, kx0, wv, ay, P.ldh);
    });
    s.mark(5);
}

template <typename T> __device__ PersistSm<T> p2_carve(const DevPlan<T>& P, const PersistCfg& C) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PersistSm<T> s;
    s.nx = P.nx;
    s.rmax = C.rmax;
    s.twx = reinterpret_cast<cplx<T>*>(smem_raw);
    s.twy = s.twx + p2_tab_len(P.nx);
    s.dpl = s.twy + p2_tab_len(P.ny);
    s.dml = s.dpl + P.ny;
    s.cdp = s.dml + P.ny;
    s.cdm = s.cdp + 8;
    s.work = s.cdm + 8;
    s.gb = s.work + p2_work_elems<T>(P.nx, P.ny, P.ldh, C.rmax, C.W);
    s.res = reinterpret_cast<T*>(s.gb + (size_t)(C.rmax / 2) * P.nx);
    s.ax = s.res + (size_t)C.nres * C.rmax * P.nx;
    s.aux = s.ax + P.nx;
    s.ay = s.aux + P.nx;
    s.auy = s.ay + ((C.rmax + 3) & ~3);
    s.kl2 = s.auy + ((C.rmax + 3) & ~3);
    s.ckx2 = s.kl2 + ((P.ny + 3) & ~3);
    s.kapt = s.ckx2 + 8;
    const int tl = (C.W * P.ny + 3) & ~3;
    s.s0t = s.kapt + tl;
    s.s1t = s.s0t + (P.lossy ? tl : 0);
    s.seg_w = s.kapt + (P.lossy ? 3 : 1) * tl;
    s.seg_i = reinterpret_cast<int*>(s.seg_w + 2 * kSegCap);
    s.flag = s.seg_i + 2 * kSegCap;
    return s;
}


// row phases of the two solves (the column phases are the SpecMode values)
enum P2Row : int {
    R_F_INIT = 0,        // p0 -> rho_xi, sample p^0, x-FFT of p^0
    R_F_U,               // u update from D+ p, x-FFT of u
    R_F_RHO_LOSSY,       // rho update from D- u, x-FFT of (rho0 div u, rho)
    R_F_RHO_LOSSLESS,    // rho update, p = c0^2 rho, sample, x-FFT of p
    R_F_P,               // p with the fractional-Laplacian terms, sample, x-FFT of p
    R_A_INIT,            // M^T h^(Nt-1) -> tail
    R_A_ABS,             // transpose of the absorption terms
    R_A_DIVT,            // transpose of e = D- u and the u update
    R_A_GRADT            // transpose of g = D+ p, M^T h^n -> tail
};

// Phase k of a solve: a column phase (col = true, SpecMode) or a row phase (P2Row), with its time
// level n.  Forward: phase 0 = R_F_INIT, then per step n = 0 .. Nt-2 the sequence GRAD, U, DIV,
// RHO (lossless) or GRAD, U, DIV, RHO, ABS, P (absorbing).  Adjoint: phase 0 = R_A_INIT, then per
// level n = Nt-2 .. 0 the sequence DIVT, A_DIVT, GRADT, A_GRADT, preceded by ABS, A_ABS when
// absorbing.
struct P2Phase {
    bool col;
    int id, n;
};
template <bool ADJ> __device__ __forceinline__ P2Phase p2_phase(int k, int Nt, bool lossy) {
    P2Phase d{false, ADJ ? (int)R_A_INIT : (int)R_F_INIT, ADJ ? Nt - 1 : 0};
    if (k == 0) return d;
    const int PP = lossy ? 6 : 4;
    const int q = (k - 1) / PP, sub = (k - 1) - q * PP;
    d.n = ADJ ? Nt - 2 - q : q;
    if (!ADJ) {
        const int col_id[6] = {SPEC_GRAD, R_F_U, SPEC_DIV, R_F_RHO_LOSSY, SPEC_ABS, R_F_P};
        d.col = (sub & 1) == 0;
        d.id = col_id[sub];
        if (!lossy && sub == 3) d.id = R_F_RHO_LOSSLESS;
    } else {
        const int ids[6] = {SPEC_ABS, R_A_ABS, SPEC_DIVT, R_A_DIVT, SPEC_GRADT, R_A_GRADT};
        const int s6 = lossy ? sub : sub + 2;
        d.col = (s6 & 1) == 0;
        d.id = ids[s6];
    }
    return d;
}

// LGX, LGY > 0: compiled for nx = 2^LGX, ny = 2^LGY (the launcher checks the plan); 0: any size
template <typename T, bool ADJ, int LGX = 0, int LGY = 0>
__global__ void __launch_bounds__(256) k_persist2(DevPlan<T> P, PersistCfg C, unsigned* gbar) {
    PersistSm<T> s = p2_carve<T>(P, C);
    const int nx = LGX ? (1 << LGX) : P.nx, ny = LGY ? (1 << LGY) : P.ny, b = blockIdx.x;
    const unsigned G = gridDim.x;
    const int pair0 = b * C.ppc;
    const int npair = max(0, min(ny / 2 - pair0, C.ppc));
    const int R = 2 * npair, line0 = 2 * pair0;
    const bool rows = R > 0, tile = b < C.ntiles;
    const int kx0 = b * C.W;
    const T dt = P.dt;
    const int Nt = P.Nt, Ns = P.sens.Ns;
    const auto axx = P2Sel<LGX>::make(P.fx.lgn);
    const auto axy = P2Sel<LGY>::make(P.fy.lgn);
    unsigned kbar = 0;
    const TraceRef TR{P.trace, P.trace_k0, P.trace_nk};
    s.tr = TR;
    s.kb = &kbar;
    cplx<T>* const A = s.work;
    cplx<T>* const B = s.work + (size_t)s.rmax * nx + p2_field_pad<T>();
    const int lgnp = (C.ppc == 1) ? 0 : (C.ppc == 2 ? 1 : (C.ppc == 4 ? 2 : 3));

    // ---- setup: stage twiddle tables, k-space tables of the tile, resident medium ----
    stage16(s.twx, P.stw[0], (size_t)p2_tab_len(nx) * sizeof(cplx<T>));
    stage16(s.twy, P.stw[1], (size_t)p2_tab_len(ny) * sizeof(cplx<T>));
    stage16(s.dpl, P.dp[1], (size_t)ny * sizeof(cplx<T>));
    stage16(s.dml, P.dm[1], (size_t)ny * sizeof(cplx<T>));
    stage_elems(s.ax, P.a[0], nx);
    stage_elems(s.aux, P.au[0], nx);
    if (threadIdx.x < (unsigned)C.W && tile) {
        const int kx = min(kx0 + (int)threadIdx.x, P.nxh - 1);
        s.cdp[threadIdx.x] = P.dp[0][kx];
        s.cdm[threadIdx.x] = P.dm[0][kx];
    }
    if (tile) {
        // the same expressions the per-phase multiply would evaluate (bit-identical multipliers)
        for (int t = threadIdx.x; t < ny * C.W; t += blockDim.x) {
            const int i = t >> C.lgW, c = t & (C.W - 1);
            const T kx = P.kv[0][min(kx0 + c, P.nxh - 1)], ky = P.kv[1][i];
            const T k2 = kx * kx + ky * ky;
            s.kapt[t] = sinc_sq(P.kap_a * P.kap_a * k2) * P.invN;
            if (P.lossy) {
                s.s0t[t] = (k2 > (T)0) ? pow(k2, P.pha) * P.invN : (T)0;
                s.s1t[t] = (k2 > (T)0) ? pow(k2, P.phb) * P.invN : (T)0;
            }
        }
    }
    for (int t = threadIdx.x; t < npair * nx; t += blockDim.x) s.gb[t] = mkc<T>(0, 0);
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
            for (int j = 0; j < 4; ++j)
                for (int t = threadIdx.x; t < R * nx; t += blockDim.x) s.row(PS_U0 + j)[t] = 0;
        }
    }
    cp_commit();
    cp_wait_all();
    __syncthreads();

    auto pml_a = [&](int xi, int r, int i) { return xi == 0 ? s.ax[i] : s.ay[r]; };
    auto pml_au = [&](int xi, int r, int i) { return xi == 0 ? s.aux[i] : s.auy[r]; };
    // adjoint: M^T h is scattered into gb, which stays zero between uses (the pointwise step that
    // reads an element clears it)
    auto take_inj = [&](int r, int i) {
        T& g = slot(s.gb, r, i, nx);
        const T v = g;
        g = (T)0;
        return v;
    };
    // adjoint: p_bar of the current level at (r, i) -> the gradient (final level), else the
    // inputs of the next x-transforms
    auto tail = [&](int r, int i, T pv, bool final_, T* out) {
        const int t = r * nx + i;
        if (final_) {
            const T sr = s.row(PS_R0)[t] + s.row(PS_R1)[t];
            P.img[(size_t)(line0 + r) * nx + i] = pv + sr / ((T)2 * s.row(PS_C2)[t]);
            return;
        }
        if (P.lossy) {
            s.row(PS_RS)[t] = pv;
            out[0] = s.row(PS_C2TAU)[t] * pv;
            out[1] = s.row(PS_C2ETA)[t] * pv;
        } else {
            const T rbar = s.row(PS_C2)[t] * pv;
            const T rho0 = s.row(PS_RHO0)[t];
#pragma unroll
            for (int xi = 0; xi < 2; ++xi) {
                const T a = pml_a(xi, r, i);
                const T rb = s.row(PS_R0 + xi)[t] + rbar;
                out[xi] = -dt * rho0 * a * rb;
                s.row(PS_R0 + xi)[t] = a * a * rb;
            }
        }
    };
    // forward: rho update from e = D- u at (r, i); returns rho0, sets sum_xi rho_xi and sum_xi e_xi
    auto rho_upd = [&](int r, int i, const T* in, T& rs, T& es) {
        const int t = r * nx + i;
        const T rho0 = s.row(PS_RHO0)[t];
        rs = 0;
        es = 0;
#pragma unroll
        for (int xi = 0; xi < 2; ++xi) {
            const T e = in[xi];
            const T a = pml_a(xi, r, i);
            const T rh = a * (a * s.row(PS_R0 + xi)[t] - dt * rho0 * e);
            s.row(PS_R0 + xi)[t] = rh;
            rs += rh;
            es += e;
        }
        return rho0;
    };

    // One row phase: inverse x-transform of FI spectra, the pointwise step of `pid`, and the
    // forward x-transform of its FO outputs (unless it ends the solve); sensor sampling from gb
    // after the pointwise step, M^T h injected through gb before it.
    auto row_phase = [&](int pid, int n, bool lastph) {
        int FI = 2, FO = 2;
        bool fwd = true, gath = false, scat = false;
        switch (pid) {
            case R_F_INIT: FI = 0; FO = 1; fwd = !lastph; gath = true; break;
            case R_F_RHO_LOSSLESS:
            case R_F_P: FO = 1; fwd = !lastph; gath = true; break;
            case R_A_INIT: FI = 0; fwd = !lastph; scat = true; break;
            case R_A_GRADT: FI = 1; fwd = !lastph; scat = true; break;
            default: break;
        }
        const bool first = (n == 0);
        T* drow = P.data + (size_t)(ADJ ? n : (pid == R_F_INIT ? 0 : n + 1)) * Ns;
        cplx<T>* a = A;
        cplx<T>* bb = B;
        if (FI > 0) p2_row_stage<T>(B, P.spec, FI, R, line0, P.ldh);
        if (scat) pscatter(s, P, seg, line0, s.gb, drow);
        if (FI > 0) {
            cp_wait_all();
            __syncthreads();
            s.mark(0);
            p2_row_in<T>(A, B, FI, npair, lgnp, axx, P.ldh);
            __syncthreads();
            s.mark(1);
            a = p2_mid<T, true>(A, B, axx, s.twx, FI * npair, lgnp);
            bb = (a == A) ? B : A;
        } else {
            __syncthreads();
        }
        s.mark(2);
        auto pw = [&](int p, int j, int m, int h, auto& z, auto& o) {
            constexpr int HH = sizeof(z[0]) / sizeof(z[0][0]);
            switch (pid) {
                case R_F_INIT:
                    p2_each<T, HH, 0, 1>(p, j, m, h, z, o, [&](int r, int i, const T*, T* out) {
                        const int t = r * nx + i;
                        const T pv = s.row(PS_RS)[t];
                        const T rh = pv / ((T)2 * s.row(PS_C2)[t]);
                        s.row(PS_R0)[t] = rh;
                        s.row(PS_R1)[t] = rh;
                        slot(s.gb, r, i, nx) = pv;
                        out[0] = pv;
                    });
                    break;
                case R_F_U:
                    p2_each<T, HH, 2, 2>(p, j, m, h, z, o, [&](int r, int i, const T* in, T* out) {
                        const int t = r * nx + i;
#pragma unroll
                        for (int xi = 0; xi < 2; ++xi) {
                            const T g = in[xi];
                            const T bq = s.row(PS_B0 + xi)[t];
                            const T au = pml_au(xi, r, i);
                            const T uo = first ? (T)0.5 * dt * bq * g : s.row(PS_U0 + xi)[t];
                            const T un = au * (au * uo - dt * bq * g);
                            s.row(PS_U0 + xi)[t] = un;
                            out[xi] = un;
                        }
                    });
                    break;
                case R_F_RHO_LOSSY:
                    p2_each<T, HH, 2, 2>(p, j, m, h, z, o, [&](int r, int i, const T* in, T* out) {
                        T rs, es;
                        const T rho0 = rho_upd(r, i, in, rs, es);
                        s.row(PS_RS)[r * nx + i] = rs;
                        out[0] = rho0 * es;
                        out[1] = rs;
                    });
                    break;
                case R_F_RHO_LOSSLESS:
                    p2_each<T, HH, 2, 1>(p, j, m, h, z, o, [&](int r, int i, const T* in, T* out) {
                        T rs, es;
                        rho_upd(r, i, in, rs, es);
                        const T pv = s.row(PS_C2)[r * nx + i] * rs;
                        slot(s.gb, r, i, nx) = pv;
                        out[0] = pv;
                    });
                    break;
                case R_F_P:
                    p2_each<T, HH, 2, 1>(p, j, m, h, z, o, [&](int r, int i, const T* in, T* out) {
                        const int t = r * nx + i;
                        const T pv = s.row(PS_C2)[t] * s.row(PS_RS)[t] + s.row(PS_C2TAU)[t] * in[0] -
                                     s.row(PS_C2ETA)[t] * in[1];
                        slot(s.gb, r, i, nx) = pv;
                        out[0] = pv;
                    });
                    break;
                case R_A_INIT:
                    p2_each<T, HH, 0, 2>(p, j, m, h, z, o, [&](int r, int i, const T*, T* out) {
                        tail(r, i, take_inj(r, i), lastph, out);
                    });
                    break;
                case R_A_ABS:
                    p2_each<T, HH, 2, 2>(p, j, m, h, z, o, [&](int r, int i, const T* in, T* out) {
                        const int t = r * nx + i;
                        const T ddbar = in[0];
                        const T rbar = s.row(PS_C2)[t] * s.row(PS_RS)[t] - in[1];
                        const T rho0 = s.row(PS_RHO0)[t];
#pragma unroll
                        for (int xi = 0; xi < 2; ++xi) {
                            const T a = pml_a(xi, r, i);
                            const T rb = s.row(PS_R0 + xi)[t] + rbar;
                            out[xi] = rho0 * ddbar - dt * rho0 * a * rb;
                            s.row(PS_R0 + xi)[t] = a * a * rb;
                        }
                    });
                    break;
                case R_A_DIVT:
                    p2_each<T, HH, 2, 2>(p, j, m, h, z, o, [&](int r, int i, const T* in, T* out) {
                        const int t = r * nx + i;
#pragma unroll
                        for (int xi = 0; xi < 2; ++xi) {
                            const T bq = s.row(PS_B0 + xi)[t];
                            const T au = pml_au(xi, r, i);
                            T ub = s.row(PS_U0 + xi)[t] + in[xi];
                            T g = -dt * bq * au * ub;
                            ub = au * au * ub;
                            if (first) g += (T)0.5 * dt * bq * ub;
                            s.row(PS_U0 + xi)[t] = ub;
                            out[xi] = g;
                        }
                    });
                    break;
                default:   // R_A_GRADT
                    p2_each<T, HH, 1, 2>(p, j, m, h, z, o, [&](int r, int i, const T* in, T* out) {
                        tail(r, i, in[0] + take_inj(r, i), lastph, out);
                    });
                    break;
            }
        };
        with_radix(axx.r0, [&](auto RC) {
            p2_row_fuse<T, decltype(RC)::value>(a, bb, s.twx, axx, npair, lgnp, FI, FO, fwd, pw);
        });
        __syncthreads();
        s.mark(3);
        if (gath) pgather(s, P, seg, line0, s.gb, drow);
        if (!fwd) return;
        cplx<T>* c = p2_mid<T, false>(bb, a, axx, s.twx, FO * npair, lgnp);
        s.mark(4);
        p2_row_out<T>(c, P.spec, s.twx, axx, FO, npair, lgnp, line0, P.ldh);
        s.mark(5);
    };

    // ---- the solve: one loop over its phases, one call site per phase kind ----
    const int nph = (Nt > 1) ? 1 + (Nt - 1) * (P.lossy ? 6 : 4) : 1;
    for (int k = 0; k < nph; ++k) {
        const P2Phase d = p2_phase<ADJ>(k, Nt, P.lossy != 0);
        const bool lastph = (k == nph - 1);
        if (d.col) {
            if (tile) p2_col<T>(s, P, axy, kx0, C.W, C.lgW, d.id);
        } else if (rows) {
            row_phase(d.id, d.n, lastph);
        }
        if (!lastph && !grid_barrier(gbar, G, kbar, s.flag, TR, P.bar_extra, P.bar_limit_ns)) return;
    }
}

}  // namespace pat
