// pat_zreg.cuh -- the z passes with the k-space multiply for 3-D grids whose z-lines have 256 points,
// every line held in registers.
//
// The work of k_spec2 / k_spec16 with lax = 2 for the multiply modes (Sec. II.A: D+-_xi and kappa;
// Eq. (state): |k|^(y-2), |k|^(y-1)): forward z-transform, multiply, inverse z-transform, on the
// half-spectrum columns kx0 .. kx0 + 7 (blockIdx.x + tile0) of one y (blockIdx.y) of every field of
// the pass.  What changes is where the transform runs:
//   * the tile [field][z][8 columns] arrives in shared memory by one tensor copy per field, under the
//     64-byte swizzle (16-byte chunk j of row z sits at chunk j ^ ((z >> 1) & 3));
//   * a half-warp owns one line (field f, column c); lane t holds the 16 points z = t + 16 n;
//   * the 256-point transform is 16 x 16: a 16-point DFT in registers, the twiddle W256^(t k), a
//     transpose through the line's own 16 x 16 shared-memory block (element (a, b) at a 16 + (b ^ a):
//     conflict-free both ways), and a second 16-point DFT, after which lane t holds the spectrum at
//     kz = t + 16 k;
//   * the multiply acts there, in registers; the inverse runs the same steps backwards and leaves lane
//     t with z = t + 16 n again;
//   * the result goes back into the tile and out by tensor copies.
// Waits for the tensor copies are bounded as in spec_stage_tile (PAT_ETIMEOUT in the status word).
#pragma once

#include "pat_spec2.cuh"

namespace pat {

// element (row z, column c) of a field's tile of 64-byte rows under the 64-byte swizzle
__device__ __forceinline__ int zsw(int z, int c) { return z * 8 + ((((c >> 1) ^ (z >> 1)) & 3) << 1) + (c & 1); }

__device__ __forceinline__ void tma_store_3d(const void* tmap, int c0, int c1, int c2, const void* src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(src);
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];\n" ::"l"(tmap),
                 "r"(c0), "r"(c1), "r"(c2), "r"(s)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// forward 256-point transform of a line held as v[n] = x[t + 16 n]; afterwards v[k] = X[t + 16 k].
// twl[k 16 + t] = W256^(t k): lanes read consecutive entries (no bank conflicts)
__device__ __forceinline__ void zfwd(float2 (&v)[16], int t, float2* tb, const float2* twl) {
    dft<float, 16, false>(v);
#pragma unroll
    for (int k = 1; k < 16; ++k) v[k] = cmul(v[k], twl[k * 16 + t]);
#pragma unroll
    for (int k = 0; k < 16; ++k) tb[t * 16 + (k ^ t)] = v[k];
    __syncwarp();
#pragma unroll
    for (int a = 0; a < 16; ++a) v[a] = tb[a * 16 + (t ^ a)];
    __syncwarp();
    dft<float, 16, false>(v);
}
// inverse (unnormalised) of a line held as v[k] = X[t + 16 k]; afterwards v[n] = x[t + 16 n]
__device__ __forceinline__ void zinv(float2 (&v)[16], int t, float2* tb, const float2* twl) {
    dft<float, 16, true>(v);
#pragma unroll
    for (int k = 1; k < 16; ++k) v[k] = cmulc(v[k], twl[k * 16 + t]);
#pragma unroll
    for (int k = 0; k < 16; ++k) tb[t * 16 + (k ^ t)] = v[k];
    __syncwarp();
#pragma unroll
    for (int a = 0; a < 16; ++a) v[a] = tb[a * 16 + (t ^ a)];
    __syncwarp();
    dft<float, 16, true>(v);
}

template <int MODE> struct ZregDims {
    static constexpr int FI = (MODE == SPEC_GRAD) ? 1 : (MODE == SPEC_ABS ? 2 : 3);
    static constexpr int FO = (MODE == SPEC_GRADT) ? 1 : (MODE == SPEC_ABS ? 2 : 3);
    static constexpr int NF = FI > FO ? FI : FO;   // fields the tile holds; 128 threads (8 lines) each
};
// shared memory: tile [NF][256][8] | transpose blocks [8 NF][16][16] | twiddles [256] (the plan's,
// staged) | lane-major twiddles [16][16] | z shift [256] (complex) | z wavenumbers [256] | kappa / N of
// the tile [8][256] (real) | mbarrier
template <int MODE> __host__ __device__ constexpr size_t zreg_smem_bytes() {
    return (size_t)(ZregDims<MODE>::NF * 2048 + ZregDims<MODE>::NF * 2048 + 768) * 8 + 256 * 4 +
           (MODE == SPEC_ABS ? 0 : 2048 * 4) + 16;
}

template <int MODE>
__global__ void __launch_bounds__(384) k_zreg(DevPlan<float> P) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    constexpr int FI = ZregDims<MODE>::FI, FO = ZregDims<MODE>::FO, NF = ZregDims<MODE>::NF;
    constexpr bool plus = (MODE == SPEC_GRAD || MODE == SPEC_DIVT);
    float2* stg = reinterpret_cast<float2*>(smem_raw);
    float2* tbuf = stg + NF * 2048;
    float2* tw = tbuf + NF * 2048;
    float2* twl = tw + 256;
    float2* ml = twl + 256;
    float* kl = reinterpret_cast<float*>(ml + 256);
    float* kap_s = kl + 256;   // (none for ABS)
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(kap_s + (MODE == SPEC_ABS ? 0 : 2048));
    const int kx0 = (blockIdx.x + P.tile0) * 8, outer = blockIdx.y;
    const int h = threadIdx.x >> 4, t = threadIdx.x & 15;
    const char* maps = static_cast<const char*>(P.tmaps) + 6 * 128;   // the swizzled z-pass maps

    // the hardware swizzle follows shared-memory address bits: the tile must start on 512 bytes
    if ((((unsigned)__cvta_generic_to_shared(stg)) & 511u) != 0) {
        if (threadIdx.x == 0 && P.fault) atomicExch(P.fault, (unsigned)PAT_EUNSUPPORTED);
        return;
    }
    // prologue: plan constants (twiddles exp(-2 pi i m / 256), the z axis' k and shift symbol)
    stage16(tw, P.twz, 256 * sizeof(float2));
    stage_elems(kl, P.kv[2], 256);
    if constexpr (MODE != SPEC_ABS) stage16(ml, plus ? P.dp[2] : P.dm[2], 256 * sizeof(float2));
    cp_commit();
    if (threadIdx.x == 0) mbar_init(bar, 1);
    pdl_trigger();
    pdl_wait();
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_expect_tx(bar, (unsigned)(FI * 2048 * sizeof(float2)));
        for (int f = 0; f < FI; ++f) tma_load_3d(stg + f * 2048, maps + f * 128, 2 * kx0, outer, 0, bar);
    }
    cp_wait_all();
    const bool ok = mbar_wait(bar, 0, 1u << 22);
    if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0 && P.fault) atomicExch(P.fault, (unsigned)PAT_ETIMEOUT);
        mbar_wait(bar, 0, 1u << 22);
        return;
    }

    // lane-major twiddles, and kappa / N of the tile's (kx, ky, kz) once for all its lines
    for (int i = threadIdx.x; i < 256; i += blockDim.x) twl[i] = tw[((i & 15) * (i >> 4)) & 255];
    if constexpr (MODE != SPEC_ABS) {
        const float ky = P.kv[1][outer];
        for (int i = threadIdx.x; i < 2048; i += blockDim.x) {
            const int cc = i >> 8, m = i & 255;
            const float kxv = P.kv[0][min(kx0 + cc, P.nxh - 1)], k = kl[m];
            kap_s[i] = sinc_sq(P.kap_a * P.kap_a * (kxv * kxv + k * k + ky * ky)) * P.invN;
        }
    }
    __syncthreads();

    // the multiply's column constants (padding columns take the last valid kx; their data are zero)
    const int c = h & 7;
    const int kx = min(kx0 + c, P.nxh - 1);
    const float kxv = P.kv[0][kx], ky = P.kv[1][outer];
    const float ckx2 = kxv * kxv, ko2 = ky * ky;
    const float2 mx = plus ? P.dp[0][kx] : P.dm[0][kx];
    const float2 mo = plus ? P.dp[1][outer] : P.dm[1][outer];
    float2* tb = tbuf + h * 256;
    auto k2_at = [&](int m) { const float k = kl[m]; return ckx2 + k * k + ko2; };
    auto kap_at = [&](int m) { return kap_s[c * 256 + m]; };
    float2 v[16];

    if constexpr (MODE == SPEC_DIV || MODE == SPEC_DIVT || MODE == SPEC_ABS) {
        const int f = h >> 3;
#pragma unroll
        for (int n = 0; n < 16; ++n) v[n] = stg[f * 2048 + zsw(t + 16 * n, c)];
        zfwd(v, t, tb, twl);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int m = t + 16 * k;
            if constexpr (MODE == SPEC_ABS) {
                const float k2 = k2_at(m);
                const float s = (f == 0) ? abs_mult0(P, k2) : ((k2 > 0.f) ? powf(k2, P.phb) * P.invN : 0.f);
                v[k] = cscale(v[k], s);
            } else {
                const float kap = kap_at(m);
                const float2 mf = (f == 0) ? mx : (f == 1 ? mo : ml[m]);
                v[k] = cscale(cmul(v[k], mf), (MODE == SPEC_DIVT) ? -kap : kap);
            }
        }
        zinv(v, t, tb, twl);
#pragma unroll
        for (int n = 0; n < 16; ++n) stg[f * 2048 + zsw(t + 16 * n, c)] = v[n];
    } else if constexpr (MODE == SPEC_GRAD) {
        // forward transform of the one input by the first 8 lines, spectrum back into its column
        if (h < 8) {
#pragma unroll
            for (int n = 0; n < 16; ++n) v[n] = stg[zsw(t + 16 * n, c)];
            zfwd(v, t, tb, twl);
#pragma unroll
            for (int k = 0; k < 16; ++k) stg[zsw(t + 16 * k, c)] = v[k];
        }
        __syncthreads();
        // output f = h >> 3: D+-_f kappa times the spectrum, inverse transform
        const int f = h >> 3;
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = stg[zsw(t + 16 * k, c)];
        __syncthreads();   // every output line has read the spectrum before any overwrites field 0
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int m = t + 16 * k;
            const float2 mf = (f == 0) ? mx : (f == 1 ? mo : ml[m]);
            v[k] = cmul(cscale(v[k], kap_at(m)), mf);
        }
        zinv(v, t, tb, twl);
#pragma unroll
        for (int n = 0; n < 16; ++n) stg[f * 2048 + zsw(t + 16 * n, c)] = v[n];
    } else {   // SPEC_GRADT: out = -kappa sum_f D+-_f in_f
        const int f = h >> 3;
#pragma unroll
        for (int n = 0; n < 16; ++n) v[n] = stg[f * 2048 + zsw(t + 16 * n, c)];
        zfwd(v, t, tb, twl);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int m = t + 16 * k;
            const float2 mf = (f == 0) ? mx : (f == 1 ? mo : ml[m]);
            stg[f * 2048 + zsw(m, c)] = cmul(v[k], mf);
        }
        __syncthreads();
        if (h < 8) {
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const int m = t + 16 * k;
                float2 a = stg[zsw(m, c)];
                a = cadd(a, stg[2048 + zsw(m, c)]);
                a = cadd(a, stg[4096 + zsw(m, c)]);
                v[k] = cscale(a, -kap_at(m));
            }
            zinv(v, t, tb, twl);
#pragma unroll
            for (int n = 0; n < 16; ++n) stg[zsw(t + 16 * n, c)] = v[n];
        }
    }
    // out: make the tile's shared-memory writes visible to the tensor copies, then store
    fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int f = 0; f < FO; ++f) tma_store_3d(maps + f * 128, 2 * kx0, outer, 0, stg + f * 2048);
        bulk_commit();
        bulk_wait_read();
    }
}

}  // namespace pat
