// pat_spec16.cuh -- spectral kernels of the per-phase path for 3-D lines of 128 and 256 points, on
// a two-stage schedule.
//
// The work of k_spec2 (pat_spec2.cuh): transforms of half-spectrum columns along y (lax = 1) or z
// (lax = 2), with the k-space multiply of Sec. II.A fused between the forward and the inverse
// transform.  The schedule differs: n = R1 x 16 (R1 = n / 16: 8 for 128 points, 16 for 256),
// forward radices (R1, 16), inverse radices (16, R1).  A transform is then two shared-memory
// passes instead of three, and a transform-multiply-transform three instead of five:
//   * stage 0 (radix R1 forward, or 16 inverse) reads the staged tile;
//   * the last forward stage (radix 16, span R1), the multiply and the first inverse stage
//     (radix 16) act on the same elements {j + r n / 16} in registers, a thread per field;
//   * the last stage (radix R1 inverse, or 16 forward) stores the spectra in natural order.
// Stage tables (p2x_stage_table): the forward radix-16 stage [15][R1] at 0, the inverse radix-R1
// stage [R1 - 1][16] after it.  Smem layout, staging, line padding and tile widths are k_spec2's.
#pragma once

#include "pat_spec2.cuh"

namespace pat {

// Last forward stage (radix 16), the k-space multiply of MODE on D fields, first inverse stage
// (radix 16); a thread takes one field (one output field for GRAD) of a butterfly.  Symbols as in
// s2_fuse.
template <typename T, int D, int MODE, class AX>
__device__ void s16_fuse(const DevPlan<T>& P, const cplx<T>* src, cplx<T>* dst, const cplx<T>* twl, const T* kl_s,
                         const cplx<T>* ml_s, int W, int lgW, const AX& ay, int lax, int kx0, int outer) {
    constexpr int FI = (MODE == SPEC_GRAD) ? 1 : (MODE == SPEC_ABS ? 2 : D);
    constexpr int FO = (MODE == SPEC_GRADT) ? 1 : (MODE == SPEC_ABS ? 2 : D);
    constexpr bool plus = (MODE == SPEC_GRAD || MODE == SPEC_DIVT);
    constexpr int R = 16;
    const int n = ay.n, m = n / R;
    const int lp = spec2_line_pad<T>();
    // work items: (field, column, butterfly) for the field-wise modes, (output field, column,
    // butterfly) for GRAD (each output redoes the one forward transform), (column, butterfly) for
    // GRADT (the sum over input fields stays in one thread)
    constexpr int NPAR = (MODE == SPEC_GRADT) ? 1 : (MODE == SPEC_GRAD ? FO : FI);
    const int lgm = ay.lg - 4, lgwm = lgW + lgm;
    for (int t = threadIdx.x; t < (NPAR << lgwm); t += blockDim.x) {
        const int q = t >> lgwm, u = t & ((1 << lgwm) - 1);
        const int c = u & (W - 1), j = u >> lgW;
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
        // multiplier of element r (i = j + r m): the same expressions as s2_fuse
        auto kap_at = [&](int r) {
            const int i = j + r * m;
            const T kl = kl_s[i];
            const T k2 = ckx2 + kl * kl + ko2;
            return sinc_sq(P.kap_a * P.kap_a * k2) * P.invN;
        };
        auto shift_at = [&](int f, int r) {
            const cplx<T> ml = ml_s[j + r * m];
            return f == 0 ? mx : (f == 1 ? ((lax == 2) ? mo : ml) : ml);
        };
        cplx<T> z[R];
        if constexpr (MODE == SPEC_GRAD) {
            p2_load<T, R, false, true>(z, src + lbase<T>(c, n, lgW, lp), j, m, m, twl);
            dft<T, R, false>(z);
#pragma unroll
            for (int r = 0; r < R; ++r) z[r] = cmul(cscale(z[r], kap_at(r)), shift_at(q, r));
            dft<T, R, true>(z);
            p2_store<T, R, true>(dst + lbase<T>(q * W + c, n, lgW, lp), j, 1, z);
        } else if constexpr (MODE == SPEC_GRADT) {
            cplx<T> acc[R];
#pragma unroll
            for (int r = 0; r < R; ++r) acc[r] = mkc<T>(0, 0);
#pragma unroll 1
            for (int f = 0; f < FI; ++f) {
                p2_load<T, R, false, true>(z, src + lbase<T>(f * W + c, n, lgW, lp), j, m, m, twl);
                dft<T, R, false>(z);
#pragma unroll
                for (int r = 0; r < R; ++r) acc[r] = cadd(acc[r], cmul(z[r], shift_at(f, r)));
            }
#pragma unroll
            for (int r = 0; r < R; ++r) acc[r] = cscale(acc[r], -kap_at(r));
            dft<T, R, true>(acc);
            p2_store<T, R, true>(dst + lbase<T>(c, n, lgW, lp), j, 1, acc);
        } else {
            const int f = q;
            p2_load<T, R, false, true>(z, src + lbase<T>(f * W + c, n, lgW, lp), j, m, m, twl);
            dft<T, R, false>(z);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if constexpr (MODE == SPEC_ABS) {
                    const int i = j + r * m;
                    const T kl = kl_s[i];
                    const T k2 = ckx2 + kl * kl + ko2;
                    const T sc = (f == 0) ? abs_mult0(P, k2) : ((k2 > (T)0) ? pow(k2, P.phb) * P.invN : (T)0);
                    z[r] = cscale(z[r], sc);
                } else {
                    const T kap = kap_at(r);
                    const T sg = (MODE == SPEC_DIVT) ? -kap : kap;
                    z[r] = cscale(cmul(z[r], shift_at(f, r)), sg);
                }
            }
            dft<T, R, true>(z);
            p2_store<T, R, true>(dst + lbase<T>(f * W + c, n, lgW, lp), j, 1, z);
        }
    }
}

// LG = 7 or 8 (128 or 256 points); D = 3
template <typename T, int D, int MODE, int LG>
__global__ void __launch_bounds__(384) k_spec16(DevPlan<T> P, int W, int lgW, int lax, int F) {
    static_assert(LG == 7 || LG == 8, "two-stage schedule for 128 or 256 points");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    constexpr bool MUL = (MODE != SPEC_PLAIN_FWD && MODE != SPEC_PLAIN_INV);
    constexpr int L = 1 << LG, R1 = L / 16;
    const int fin = (MODE == SPEC_GRAD) ? 1 : (MODE == SPEC_ABS ? 2 : (MUL ? D : F));
    const int fout = (MODE == SPEC_GRADT) ? 1 : (MODE == SPEC_ABS ? 2 : (MUL ? D : F));
    const P2AxisC<LG> ay{};
    cplx<T>* tab = reinterpret_cast<cplx<T>*>(smem_raw);
    cplx<T>* ml_s = tab + p2_tab_len(L);
    T* kl_s = reinterpret_cast<T*>(ml_s + L);
    cplx<T>* A = tab + spec2_pre_elems<T>(L);
    cplx<T>* B = A + spec2_buf_elems<T>(spec2_nf(D, MODE, F), L, W);
    const cplx<T>* tw_f = tab;               // forward radix-16 stage, span R1
    const cplx<T>* tw_i = tab + 15 * R1;     // inverse radix-R1 stage, span 16
    const int kx0 = (blockIdx.x + P.tile0) * W, outer = blockIdx.y;
    const int wv = min(W, P.nxh - kx0);
    const size_t es = (lax == 1) ? (size_t)P.ldh : (size_t)P.ny * P.ldh;
    const size_t base = (lax == 1) ? (size_t)outer * P.ny * P.ldh + kx0 : (size_t)outer * P.ldh + kx0;

    // prologue: stage tables and the line axis' k-space data (plan constants)
    stage16(tab, P.stw16[lax], (size_t)p2_tab_len(L) * sizeof(cplx<T>));
    if constexpr (MUL) {
        constexpr bool plus = (MODE == SPEC_GRAD || MODE == SPEC_DIVT);
        stage_elems(kl_s, P.kv[lax], L);
        if constexpr (MODE != SPEC_ABS) stage16(ml_s, plus ? P.dp[lax] : P.dm[lax], (size_t)L * sizeof(cplx<T>));
    }
    pdl_trigger();
    pdl_wait();
    // stage the tile's columns of every input field: B[f][i][c] (k_spec2's staging)
    if (!spec_stage_tile(P, B, fin, L, W, lgW, lax, kx0, outer, base, es)) return;

    if constexpr (MODE == SPEC_PLAIN_INV) {
        s2_in<T, 16, true>(A, B, fin, W, lgW, ay);
        __syncthreads();
        s2_out<T, R1, true>(A, P.spec, tw_i, fout, W, lgW, wv, ay, base, es);
    } else {
        s2_in<T, R1, false>(A, B, fin, W, lgW, ay);
        __syncthreads();
        if constexpr (!MUL) {
            s2_out<T, 16, false>(A, P.spec, tw_f, fout, W, lgW, wv, ay, base, es);
        } else {
            s16_fuse<T, D, MODE>(P, A, B, tw_f, kl_s, ml_s, W, lgW, ay, lax, kx0, outer);
            __syncthreads();
            s2_out<T, R1, true>(B, P.spec, tw_i, fout, W, lgW, wv, ay, base, es);
        }
    }
}

}  // namespace pat
