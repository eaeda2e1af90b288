// pat_spec2.cuh -- spectral kernels of the per-phase path for power-of-two line lengths.
//
// The same work as k_spec (pat_kernels.cuh): transforms of half-spectrum columns along y (lax = 1)
// or z (lax = 2), with the k-space multiply of Sec. II.A / Eq. (state) fused between the forward and
// the inverse transform for the multiply modes.  What changes is the transform, which follows the
// fixed power-of-two Stockham schedule of the persistent kernel (pat_persist2.cuh):
//   * the tile's columns are staged with cp.async into the spare line buffer, and the first stage
//     reads them from there;
//   * the last forward stage, the k-space multiply and the first inverse stage run in registers on
//     the same elements {j + r L/8};
//   * the last stage stores straight to the spectra in natural order;
//   * lines are XOR-swizzled and 16 bytes apart beyond their length (lanes step across the tile's
//     lines), fields another 64 bytes apart, twiddles per stage.
// A tile is W columns x F fields (W <= 8: ceil((nx/2 + 1) / W) W must not pass the padded row ldh);
// shared memory holds max(fields in, fields out) of them (spec2_nf), sized per launch.
#pragma once

#include "pat_persist2.cuh"

namespace pat {

// Stage the tile's columns of the fin input fields into B[f][i][c] (dense, W columns per line; tiles
// reach into the zeroed padding columns of the half spectra, kx0 + W <= ldh).  With the plan's tensor
// maps (FP32, W = 8 columns: 64-byte rows; lines of at most 256 points), one thread issues one tensor
// copy per field onto an mbarrier that counts the bytes, and the CTA waits for them; otherwise every
// thread issues 16-byte cp.async copies.  The wait is bounded: when it runs out the status word gets
// PAT_ETIMEOUT, the CTA waits (bounded again) for the copies in flight and the function returns
// false in every thread, and the caller returns.
template <typename T>
__device__ __forceinline__ bool spec_stage_tile(const DevPlan<T>& P, cplx<T>* B, int fin, int L, int W, int lgW,
                                                int lax, int kx0, int outer, size_t base, size_t es) {
    __shared__ unsigned long long tma_bar;
    const bool tma = sizeof(T) == 4 && P.use_tma && W == 8 && L <= 256 &&
                     (((unsigned)__cvta_generic_to_shared(B)) & 127u) == 0;
    if (tma) {
        if (threadIdx.x == 0) mbar_init(&tma_bar, 1);
        __syncthreads();
        if (threadIdx.x == 0) {
            mbar_expect_tx(&tma_bar, (unsigned)((size_t)fin * L * W * sizeof(cplx<T>)));
            const char* maps = static_cast<const char*>(P.tmaps) + (lax == 1 ? 0 : 3) * 128;
            for (int f = 0; f < fin; ++f)
                tma_load_3d(B + (size_t)f * L * W, maps + f * 128, 2 * kx0, lax == 1 ? 0 : outer, lax == 1 ? outer : 0,
                            &tma_bar);
        }
        const bool ok = mbar_wait(&tma_bar, 0, 1u << 22);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0 && P.fault) atomicExch(P.fault, (unsigned)PAT_ETIMEOUT);
            mbar_wait(&tma_bar, 0, 1u << 22);
            return false;
        }
        return true;
    }
    const int cb = W * (int)sizeof(cplx<T>);
    for (int f = 0; f < fin; ++f) {
        const cplx<T>* src = P.spec[f] + base;
        cplx<T>* d = B + f * L * W;
        if (cb >= 16) {
            constexpr int EPC = 16 / (int)sizeof(cplx<T>);
            const int cpr = cb / 16, lgc = lgW - (EPC == 2 ? 1 : 0);   // 16-byte pieces per row: 2^lgc
            for (int t = threadIdx.x; t < L * cpr; t += blockDim.x) {
                const int i = t >> lgc, ch = t & (cpr - 1);
                cp_async<16>(d + i * W + ch * EPC, src + (size_t)i * es + ch * EPC);
            }
        } else {
            for (int i = threadIdx.x; i < L; i += blockDim.x) cp_async<sizeof(cplx<T>)>(d + i, src + (size_t)i * es);
        }
    }
    cp_commit();
    cp_wait_all();
    __syncthreads();
    return true;
}

// stage 0 (radix R, no twiddles; forward or inverse) from the staged tile S[f][i][c]
template <typename T, int R, bool INV, class AX>
__device__ void s2_in(cplx<T>* dst, const cplx<T>* S, int FI, int W, int lgW, const AX& ay) {
    const int n = ay.n, lgm = ay.lg - Lg2<R>::v, m = 1 << lgm;
    for (int t = threadIdx.x; t < ((FI * W) << lgm); t += blockDim.x) {
        const int c = t & (W - 1), j = (t >> lgW) & (m - 1), f = t >> (lgW + lgm);
        const cplx<T>* src = S + (f * n + j) * W + c;   // staged tile [f][i][c], i = j + r m
        const int step = m * W;
        cplx<T> v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src[r * step];
        dft<T, R, INV>(v);
        p2_store<T, R, P2IsC<AX>::value>(dst + lbase<T>(f * W + c, n, lgW, spec2_line_pad<T>()), j, 1, v);
    }
}

// last stage (radix R, span n / R; forward or inverse) and the store of valid columns
template <typename T, int R, bool INV, class AX>
__device__ void s2_out(const cplx<T>* src, cplx<T>* const* spec, const cplx<T>* twl, int FO, int W, int lgW,
                       int wv, const AX& ay, size_t base, size_t es) {
    const int n = ay.n, lgm = ay.lg - Lg2<R>::v, m = 1 << lgm;
    for (int t = threadIdx.x; t < ((FO * W) << lgm); t += blockDim.x) {
        const int c = t & (W - 1), j = (t >> lgW) & (m - 1), f = t >> (lgW + lgm);
        cplx<T> v[R];
        p2_load<T, R, INV, P2IsC<AX>::value>(v, src + lbase<T>(f * W + c, n, lgW, spec2_line_pad<T>()), j, m, m,
                                             twl);
        dft<T, R, INV>(v);
        if (c < wv) {
            cplx<T>* dst = spec[f] + base + c + (size_t)j * es;
            const size_t mes = (size_t)m * es;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                *dst = v[r];
                dst += mes;
            }
        }
    }
}

// Last forward stage (radix 8), the k-space multiply of MODE on D fields, first inverse stage.
// Symbols (Sec. II.A, Eq. (state)): kappa = sinc(c_ref |k| dt / 2), D+-_xi = i k_xi e^{+-i k_xi h/2},
// |k|^(y-2), |k|^(y-1); all scaled by 1/N.  Field f's shift factor: f = 0 -> x (column kx),
// f = 1 -> y (the CTA's outer index in a z pass, the line index in a y pass), f = 2 -> z (line).
template <typename T, int D, int MODE, class AX>
__device__ void s2_fuse(const DevPlan<T>& P, const cplx<T>* src, cplx<T>* dst, const cplx<T>* twl, const T* kl_s,
                        const cplx<T>* ml_s, int W, int lgW, const AX& ay, int lax, int kx0, int outer) {
    constexpr bool CM = P2IsC<AX>::value;
    constexpr int FI = (MODE == SPEC_GRAD) ? 1 : (MODE == SPEC_ABS ? 2 : D);
    constexpr int FO = (MODE == SPEC_GRADT) ? 1 : (MODE == SPEC_ABS ? 2 : D);
    constexpr bool plus = (MODE == SPEC_GRAD || MODE == SPEC_DIVT);
    const int n = ay.n, lgm = ay.lg - 3, m = 1 << lgm;
    for (int t = threadIdx.x; t < (W << lgm); t += blockDim.x) {
        const int c = t & (W - 1), j = t >> lgW;
        cplx<T> z[FI][8];
#pragma unroll
        for (int f = 0; f < FI; ++f) {
            p2_load<T, 8, false, CM>(z[f], src + lbase<T>(f * W + c, n, lgW, spec2_line_pad<T>()), j, m, m, twl);
            dft<T, 8, false>(z[f]);
        }
        const int kx = min(kx0 + c, P.nxh - 1);
        const T kxv = P.kv[0][kx];
        const T ckx2 = kxv * kxv;
        T ko2 = 0;
        cplx<T> mo = mkc<T>(0, 0);
        if (lax == 2) {
            const T ky = P.kv[1][outer];
            ko2 = ky * ky;
            mo = plus ? P.dp[1][outer] : P.dm[1][outer];
        }
        const cplx<T> mx = plus ? P.dp[0][kx] : P.dm[0][kx];
        cplx<T> o[FO][8];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int i = j + r * m;
            const T kl = kl_s[i];
            const T k2 = ckx2 + kl * kl + ko2;
            if constexpr (MODE == SPEC_ABS) {
                const T s0 = abs_mult0(P, k2);
                const T s1 = (k2 > (T)0) ? pow(k2, P.phb) * P.invN : (T)0;
                o[0][r] = cscale(z[0][r], s0);
                o[FO - 1][r] = cscale(z[FI - 1][r], s1);
            } else {
                const T kap = sinc_sq(P.kap_a * P.kap_a * k2) * P.invN;
                const T sg = (MODE == SPEC_DIVT || MODE == SPEC_GRADT) ? -kap : kap;
                const cplx<T> ml = ml_s[i];
                cplx<T> mf[3];
                mf[0] = mx;
                mf[1] = (lax == 2) ? mo : ml;
                mf[2] = ml;
                if constexpr (MODE == SPEC_GRAD) {
                    const cplx<T> v = cscale(z[0][r], sg);
#pragma unroll
                    for (int f = 0; f < FO; ++f) o[f][r] = cmul(v, mf[f]);
                } else if constexpr (MODE == SPEC_GRADT) {
                    cplx<T> acc = mkc<T>(0, 0);
#pragma unroll
                    for (int f = 0; f < FI; ++f) acc = cadd(acc, cmul(z[f][r], mf[f]));
                    o[0][r] = cscale(acc, sg);
                } else {
#pragma unroll
                    for (int f = 0; f < FO; ++f) o[f][r] = cscale(cmul(z[f][r], mf[f]), sg);
                }
            }
        }
#pragma unroll
        for (int g = 0; g < FO; ++g) {
            dft<T, 8, true>(o[g]);
            p2_store<T, 8, CM>(dst + lbase<T>(g * W + c, n, lgW, spec2_line_pad<T>()), j, 1, o[g]);
        }
    }
}

// LG > 0: compiled for lines of 2^LG points (the launcher checks the plan); 0: any power of two
template <typename T, int D, int MODE, int LG = 0>
__global__ void __launch_bounds__(256) k_spec2(DevPlan<T> P, int W, int lgW, int lax, int F) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    constexpr bool MUL = (MODE != SPEC_PLAIN_FWD && MODE != SPEC_PLAIN_INV);
    const int fin = (MODE == SPEC_GRAD) ? 1 : (MODE == SPEC_ABS ? 2 : (MUL ? D : F));
    const int fout = (MODE == SPEC_GRADT) ? 1 : (MODE == SPEC_ABS ? 2 : (MUL ? D : F));
    const auto ay = P2Sel<LG>::make((lax == 1) ? P.fy.lgn : P.fz.lgn);
    const int L = ay.n;
    cplx<T>* tab = reinterpret_cast<cplx<T>*>(smem_raw);
    cplx<T>* ml_s = tab + p2_tab_len(L);
    T* kl_s = reinterpret_cast<T*>(ml_s + L);
    cplx<T>* A = tab + spec2_pre_elems<T>(L);
    cplx<T>* B = A + spec2_buf_elems<T>(spec2_nf(D, MODE, F), L, W);
    const int kx0 = (blockIdx.x + P.tile0) * W, outer = blockIdx.y;
    const int wv = min(W, P.nxh - kx0);
    const size_t es = (lax == 1) ? (size_t)P.ldh : (size_t)P.ny * P.ldh;
    const size_t base = (lax == 1) ? (size_t)outer * P.ny * P.ldh + kx0 : (size_t)outer * P.ldh + kx0;

    // prologue: stage twiddle tables (plan constants, never written by the preceding kernel)
    stage16(tab, P.stw[lax], (size_t)p2_tab_len(L) * sizeof(cplx<T>));
    if constexpr (MUL) {
        // the line axis' wavenumbers and its shift operator (D+ for GRAD / DIVT, D- otherwise)
        constexpr bool plus = (MODE == SPEC_GRAD || MODE == SPEC_DIVT);
        stage_elems(kl_s, P.kv[lax], L);
        if constexpr (MODE != SPEC_ABS) stage16(ml_s, plus ? P.dp[lax] : P.dm[lax], (size_t)L * sizeof(cplx<T>));
    }
    pdl_trigger();
    pdl_wait();
    // stage the tile's columns of every input field: B[f][i][c]
    if (!spec_stage_tile(P, B, fin, L, W, lgW, lax, kx0, outer, base, es)) return;

    if constexpr (MODE == SPEC_PLAIN_INV) {
        s2_in<T, 8, true>(A, B, fin, W, lgW, ay);
        __syncthreads();
        cplx<T>* a = p2_mid<T, true>(A, B, ay, tab, fin * W, lgW, spec2_line_pad<T>());
        with_radix(ay.r0, [&](auto RC) {
            s2_out<T, decltype(RC)::value, true>(a, P.spec, tab + p2_off_i(ay, ay.nst - 1), fout, W, lgW, wv, ay,
                                                 base, es);
        });
    } else {
        with_radix(ay.r0, [&](auto RC) { s2_in<T, decltype(RC)::value, false>(A, B, fin, W, lgW, ay); });
        __syncthreads();
        cplx<T>* a = p2_mid<T, false>(A, B, ay, tab, fin * W, lgW, spec2_line_pad<T>());
        if constexpr (!MUL) {
            s2_out<T, 8, false>(a, P.spec, tab + p2_off_f(ay, ay.nst - 1), fout, W, lgW, wv, ay, base, es);
        } else {
            cplx<T>* b = (a == A) ? B : A;
            s2_fuse<T, D, MODE>(P, a, b, tab + p2_off_f(ay, ay.nst - 1), kl_s, ml_s, W, lgW, ay, lax, kx0, outer);
            __syncthreads();
            cplx<T>* r = p2_mid<T, true>(b, a, ay, tab, fout * W, lgW, spec2_line_pad<T>());
            with_radix(ay.r0, [&](auto RC) {
                s2_out<T, decltype(RC)::value, true>(r, P.spec, tab + p2_off_i(ay, ay.nst - 1), fout, W, lgW, wv, ay,
                                                     base, es);
            });
        }
    }
}

}  // namespace pat
