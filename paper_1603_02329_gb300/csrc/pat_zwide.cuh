// pat_zwide.cuh -- the z passes with the k-space multiply for 3-D grids whose z-lines have 128 or
// 256 points, on 16-column tiles transformed in place in shared memory.
//
// The work of k_spec2 / k_spec16 / k_zreg with lax = 2: forward z-transform, multiply (Sec. II.A:
// kappa D+-_xi; Eq. (state): |k|^(y-2), |k|^(y-1)), inverse z-transform, on half-spectrum columns
// kx0 .. kx0 + 15 of one ky (blockIdx.z).  The transforms take the two-stage schedule of k_ywide
// (n = R1 x 16; forward radices (R1, 16), inverse (16, R1)):
//   * a tile [z][16 columns] arrives by one tensor copy; forward stage 0 writes back in place;
//   * forward stage 1 leaves thread (j, c) with the spectrum at kz = j + R1 k, k < 16: the elements
//     on which inverse stage 0 acts, so the multiply and inverse stage 0 follow in registers; the
//     outputs go back in place once every thread has read its stage-1 inputs;
//   * inverse stage 1 reads consecutive rows and stores straight to the spectra.
// The CTA layout follows the fields:
//   * D-, its transpose and the absorption pass: every output field depends on its own input field,
//     so a CTA holds one field (blockIdx.x), and the CTAs of a tile run next to each other;
//   * D+ (one input, D outputs): one forward transform, then per output the multiply and the inverse
//     transform through the same tile buffer;
//   * the transpose of D+ (D inputs, one output): three tiles by tensor copies, the products summed in
//     registers, one inverse transform.
// The multipliers come from the plan's tables (k_kap_table, k_abs_table: the expressions of the other
// z passes, evaluated once per plan), read for the CTA's elements while the tile is in flight; the
// absorption pass computes them inline when no table applies (the time-reversal window).  Waits for
// the tensor copies are bounded as in spec_stage_tile (PAT_ETIMEOUT in the status word).
#pragma once

#include "pat_spec2.cuh"

namespace pat {

// kappa / N on the half spectrum, layout [ky][kz][ldh] (padding columns: the last valid kx), the
// expression of the z passes: sinc((c_ref dt / 2) |k|) with |k|^2 = kx^2 + kz^2 + ky^2 in that order
__global__ void k_kap_table(DevPlan<float> P, float* kap) {
    const size_t n = (size_t)P.ny * P.nz * P.ldh;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int kx = (int)(i % P.ldh);
        const size_t q = i / P.ldh;
        const int kz = (int)(q % P.nz), ky = (int)(q / P.nz);
        const float kxv = P.kv[0][min(kx, P.nxh - 1)], kl = P.kv[2][kz], kyv = P.kv[1][ky];
        const float k2 = kxv * kxv + kl * kl + kyv * kyv;
        kap[i] = sinc_sq(P.kap_a * P.kap_a * k2) * P.invN;
    }
}
// the absorption pass' multipliers without the time-reversal window, [2][ky][kz][ldh]: field 0
// |k|^(y-2) / N (the operand of tau), field 1 |k|^(y-1) / N (of eta); 0 at k = 0
__global__ void k_abs_table(DevPlan<float> P, float* tab) {
    const size_t n = (size_t)P.ny * P.nz * P.ldh;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int kx = (int)(i % P.ldh);
        const size_t q = i / P.ldh;
        const int kz = (int)(q % P.nz), ky = (int)(q / P.nz);
        const float kxv = P.kv[0][min(kx, P.nxh - 1)], kl = P.kv[2][kz], kyv = P.kv[1][ky];
        const float k2 = kxv * kxv + kl * kl + kyv * kyv;
        tab[i] = (k2 > 0.f) ? powf(k2, P.pha) * P.invN : 0.f;
        tab[n + i] = (k2 > 0.f) ? powf(k2, P.phb) * P.invN : 0.f;
    }
}

template <int MODE> struct ZwideDims {
    static constexpr int NT = (MODE == SPEC_GRADT) ? 3 : 1;   // tiles in shared memory
};
// shared memory: NT tiles [L][16] (complex) | stage tables [2 L] | z shift [L] (complex) | z
// wavenumbers [L] (real) | mbarrier
template <int MODE> __host__ __device__ constexpr size_t zwide_smem_bytes(int L) {
    return (size_t)ZwideDims<MODE>::NT * L * 16 * sizeof(float2) + (size_t)p2_tab_len(L) * sizeof(float2) +
           (size_t)L * sizeof(float2) + (size_t)L * sizeof(float) + 16;
}

// LG = 7 or 8.  grid (fields, ceil(nxh / 16), ny) for the field-wise modes, (1, ceil(nxh / 16), ny)
// for SPEC_GRAD and SPEC_GRADT; 256 threads.  mt: kappa / N ([ky][kz][ldh]) for every mode but
// SPEC_ABS, the two absorption tables or nullptr (inline) for SPEC_ABS.
template <int LG, int MODE>
__global__ void __launch_bounds__(256, (MODE == SPEC_GRADT) ? 2 : (MODE == SPEC_GRAD ? 3 : 4)) k_zwide(DevPlan<float> P, const float* __restrict__ mt) {
    static_assert(LG == 7 || LG == 8, "two-stage schedule for 128 or 256 points");
    constexpr int L = 1 << LG, R1 = L / 16, NT = ZwideDims<MODE>::NT;
    constexpr bool plus = (MODE == SPEC_GRAD || MODE == SPEC_DIVT);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float2* S = reinterpret_cast<float2*>(smem_raw);
    float2* tab = S + NT * L * 16;
    float2* ml = tab + p2_tab_len(L);
    float* kl = reinterpret_cast<float*>(ml + L);
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(kl + L);
    const float2* tw_f = tab;             // forward radix-16 stage, span R1: [15][R1]
    const float2* tw_i = tab + 15 * R1;   // inverse radix-R1 stage, span 16: [R1 - 1][16]
    const int f0 = blockIdx.x, kx0 = blockIdx.y * 16, outer = blockIdx.z;
    const int wv = min(16, P.nxh - kx0);
    const int c = threadIdx.x & 15, j = threadIdx.x >> 4;
    const size_t es = (size_t)P.ny * P.ldh;

    // a tensor copy into shared memory starts on 128 bytes
    if ((((unsigned)__cvta_generic_to_shared(S)) & 127u) != 0) {
        if (threadIdx.x == 0 && P.fault) atomicExch(P.fault, (unsigned)PAT_EUNSUPPORTED);
        return;
    }
    // prologue: plan constants (stage tables, the z axis' k and shift symbol)
    stage16(tab, P.stw16[2], (size_t)p2_tab_len(L) * sizeof(float2));
    stage_elems(kl, P.kv[2], L);
    if constexpr (MODE != SPEC_ABS) stage16(ml, plus ? P.dp[2] : P.dm[2], (size_t)L * sizeof(float2));
    cp_commit();
    if (threadIdx.x == 0) mbar_init(bar, 1);
    // the multiply's column constants (padding columns take the last valid kx; their data are zero)
    const int kx = min(kx0 + c, P.nxh - 1);
    const float kxv = P.kv[0][kx], ky = P.kv[1][outer];
    const float ckx2 = kxv * kxv, ko2 = ky * ky;
    const float2 mx = plus ? P.dp[0][kx] : P.dm[0][kx];
    const float2 mo = plus ? P.dp[1][outer] : P.dm[1][outer];
    // the multiplier of this thread's stage-1 elements kz = j + R1 k (plan constants: read before the
    // wait); field f0's absorption table
    float kp[16];
    const bool tabled = (MODE != SPEC_ABS) || mt != nullptr;
    if (tabled) {
        const float* kr = mt + (MODE == SPEC_ABS ? (size_t)f0 * P.nz * es : 0) + (size_t)outer * P.nz * P.ldh + kx0 + c;
#pragma unroll
        for (int k = 0; k < 16; ++k) kp[k] = (j < R1 && c < wv) ? __ldg(kr + (size_t)(j + R1 * k) * P.ldh) : 0.f;
    }
    pdl_trigger();
    pdl_wait();
    __syncthreads();
    if (threadIdx.x == 0) {
        const char* maps = static_cast<const char*>(P.tmaps) + 12 * 128;   // the 16-column z-pass maps
        mbar_expect_tx(bar, (unsigned)(NT * L * 16 * sizeof(float2)));
        for (int t = 0; t < NT; ++t) tma_load_3d(S + t * L * 16, maps + (f0 + t) * 128, 2 * kx0, outer, 0, bar);
    }
    cp_wait_all();
    const bool ok = mbar_wait(bar, 0, 1u << 22);
    if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0 && P.fault) atomicExch(P.fault, (unsigned)PAT_ETIMEOUT);
        mbar_wait(bar, 0, 1u << 22);
        return;
    }

    auto shift = [&](int f, int m) { return (f == 0) ? mx : (f == 1 ? mo : ml[m]); };
    // forward stage 0 of tile T, radix R1 (no twiddles): butterfly j < 16 on rows j + 16 r, in place
    auto fwd0 = [&](float2* T) {
        float2 v[R1];
#pragma unroll
        for (int r = 0; r < R1; ++r) v[r] = T[(j + 16 * r) * 16 + c];
        dft<float, R1, false>(v);
#pragma unroll
        for (int r = 0; r < R1; ++r) T[(j + 16 * r) * 16 + c] = v[r];
    };
    // forward stage 1 (radix 16, span R1) of the inputs loaded from rows r + 16 j: the spectrum at
    // kz = j + R1 k
    auto load1 = [&](const float2* T, float2(&v)[16]) {
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = T[(r + 16 * j) * 16 + c];
    };
    auto fwd1 = [&](float2(&v)[16]) {
#pragma unroll
        for (int r = 1; r < 16; ++r) v[r] = cmul(v[r], tw_f[(r - 1) * R1 + j]);
        dft<float, 16, false>(v);
    };
    // inverse stage 0 (radix 16) of the multiplied spectrum, outputs to rows j + R1 r
    auto inv0 = [&](float2* T, float2(&v)[16]) {
        dft<float, 16, true>(v);
#pragma unroll
        for (int r = 0; r < 16; ++r) T[(j + R1 * r) * 16 + c] = v[r];
    };
    // inverse stage 1, radix R1, span 16: butterfly j < 16 on rows r + R1 j, conjugate-twiddled; its
    // outputs are the line at z = j + 16 k of output field f
    auto inv1 = [&](const float2* T, int f) {
        float2 w[R1];
#pragma unroll
        for (int r = 0; r < R1; ++r) w[r] = T[(r + R1 * j) * 16 + c];
#pragma unroll
        for (int r = 1; r < R1; ++r) w[r] = cmulc(w[r], tw_i[(r - 1) * 16 + j]);
        dft<float, R1, true>(w);
        if (c < wv) {
            float2* out = P.spec[f] + (size_t)outer * P.ldh + kx0 + c;
#pragma unroll
            for (int k = 0; k < R1; ++k) out[(size_t)(j + 16 * k) * es] = w[k];
        }
    };

    float2 v[16];
    if constexpr (MODE == SPEC_DIV || MODE == SPEC_DIVT || MODE == SPEC_ABS) {
        const int f = f0;
        fwd0(S);
        __syncthreads();
        if (j < R1) load1(S, v);
        __syncthreads();
        if (j < R1) {
            fwd1(v);
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                if constexpr (MODE == SPEC_ABS) {
                    float sc = kp[k];
                    if (!tabled) {
                        const int m = j + R1 * k;
                        const float k2 = ckx2 + kl[m] * kl[m] + ko2;
                        sc = (f == 0) ? abs_mult0(P, k2) : ((k2 > 0.f) ? powf(k2, P.phb) * P.invN : 0.f);
                    }
                    v[k] = cscale(v[k], sc);
                } else {
                    v[k] = cscale(cmul(v[k], shift(f, j + R1 * k)), (MODE == SPEC_DIVT) ? -kp[k] : kp[k]);
                }
            }
            inv0(S, v);
        }
        __syncthreads();
        inv1(S, f);
    } else if constexpr (MODE == SPEC_GRAD) {
        // one forward transform of the input; per output field f: kappa D+_f, inverse transform
        fwd0(S);
        __syncthreads();
        if (j < R1) load1(S, v);
        __syncthreads();
        if (j < R1) fwd1(v);
#pragma unroll 1
        for (int f = 0; f < 3; ++f) {
            if (j < R1) {
                float2 w[16];
#pragma unroll
                for (int k = 0; k < 16; ++k) w[k] = cmul(cscale(v[k], kp[k]), shift(f, j + R1 * k));
                inv0(S, w);
            }
            __syncthreads();
            inv1(S, f);
            __syncthreads();   // every thread has read the tile before the next output overwrites it
        }
    } else {   // SPEC_GRADT: out = -kappa sum_f D-_f in_f
        fwd0(S);
        fwd0(S + L * 16);
        fwd0(S + 2 * L * 16);
        __syncthreads();
        float2 acc[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) acc[k] = make_float2(0.f, 0.f);
#pragma unroll 1
        for (int f = 0; f < 3; ++f) {
            if (j < R1) {
                load1(S + f * L * 16, v);
                fwd1(v);
#pragma unroll
                for (int k = 0; k < 16; ++k) acc[k] = cadd(acc[k], cmul(v[k], shift(f, j + R1 * k)));
            }
        }
        __syncthreads();   // every stage-1 read of tile 0 is done before inverse stage 0 writes it
        if (j < R1) {
#pragma unroll
            for (int k = 0; k < 16; ++k) acc[k] = cscale(acc[k], -kp[k]);
            inv0(S, acc);
        }
        __syncthreads();
        inv1(S, 0);
    }
}

}  // namespace pat
