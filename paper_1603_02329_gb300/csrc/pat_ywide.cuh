// pat_ywide.cuh -- the plain y transforms of 3-D grids whose y-lines have 128 or 256 points: one
// field of a 16-column tile per CTA, transformed in place in the staged tile.
//
// The work of k_spec16 with MODE = SPEC_PLAIN_FWD / SPEC_PLAIN_INV and lax = 1 (the y passes around
// every k-space multiply of Sec. II.A), with the same operations: n = R1 x 16 (R1 = n / 16), forward
// radices (R1, 16), inverse radices (16, R1), the same stage tables, butterflies and twiddle products
// (the compiler contracts them into fused multiply-adds its own way, so results differ from k_spec16's
// in the last bits: 3e-7 to 4e-7 relative over a solve).  What changes is the data movement:
//   * a tile is 16 half-spectrum columns wide (rows of 128 bytes, whole cache lines) and holds one
//     field (blockIdx.z); it arrives by one tensor copy;
//   * the first stage writes each butterfly's outputs back to the slots it read (in place), so the
//     tile is the only buffer;
//   * the second stage reads its inputs from consecutive rows of the tile and stores its outputs
//     straight to the spectra: one store instruction of a warp writes two 128-byte rows.
// Thread (j, c) = (threadIdx.x >> 4, threadIdx.x & 15) runs butterfly j of column c.  Waits for the
// tensor copy are bounded as in spec_stage_tile (PAT_ETIMEOUT in the status word).
#pragma once

#include "pat_spec2.cuh"

namespace pat {

// shared memory: tile [L][16] (complex) | stage tables [2 L] | mbarrier
__host__ __device__ constexpr size_t ywide_smem_bytes(int L) {
    return (size_t)L * 16 * sizeof(float2) + (size_t)p2_tab_len(L) * sizeof(float2) + 16;
}

// LG = 7 or 8; INV: the inverse transform.  grid (ceil(nxh / 16), nz, fields), 256 threads.
template <int LG, bool INV>
__global__ void __launch_bounds__(256) k_ywide(DevPlan<float> P) {
    static_assert(LG == 7 || LG == 8, "two-stage schedule for 128 or 256 points");
    constexpr int L = 1 << LG, R1 = L / 16;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float2* S = reinterpret_cast<float2*>(smem_raw);
    float2* tab = S + L * 16;
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(tab + p2_tab_len(L));
    const float2* tw_f = tab;             // forward radix-16 stage, span R1: [15][R1]
    const float2* tw_i = tab + 15 * R1;   // inverse radix-R1 stage, span 16: [R1 - 1][16]
    const int kx0 = blockIdx.x * 16, outer = blockIdx.y, f = blockIdx.z;
    const int wv = min(16, P.nxh - kx0);
    const int c = threadIdx.x & 15, j = threadIdx.x >> 4;

    // a tensor copy into shared memory starts on 128 bytes
    if ((((unsigned)__cvta_generic_to_shared(S)) & 127u) != 0) {
        if (threadIdx.x == 0 && P.fault) atomicExch(P.fault, (unsigned)PAT_EUNSUPPORTED);
        return;
    }
    // prologue: the stage tables (plan constants)
    stage16(tab, P.stw16[1], (size_t)p2_tab_len(L) * sizeof(float2));
    cp_commit();
    if (threadIdx.x == 0) mbar_init(bar, 1);
    pdl_trigger();
    pdl_wait();
    __syncthreads();
    if (threadIdx.x == 0) {
        const char* maps = static_cast<const char*>(P.tmaps) + 9 * 128;   // the 16-column y-pass maps
        mbar_expect_tx(bar, (unsigned)(L * 16 * sizeof(float2)));
        tma_load_3d(S, maps + f * 128, 2 * kx0, 0, outer, bar);
    }
    cp_wait_all();
    const bool ok = mbar_wait(bar, 0, 1u << 22);
    if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0 && P.fault) atomicExch(P.fault, (unsigned)PAT_ETIMEOUT);
        mbar_wait(bar, 0, 1u << 22);
        return;
    }

    float2* out = P.spec[f] + (size_t)outer * P.ny * P.ldh + kx0 + c;
    const size_t es = (size_t)P.ldh;
    if constexpr (!INV) {
        // stage 0, radix R1 (no twiddles): butterfly j < 16 on rows j + 16 r, outputs back in place
        {
            float2 v[R1];
#pragma unroll
            for (int r = 0; r < R1; ++r) v[r] = S[(j + 16 * r) * 16 + c];
            dft<float, R1, false>(v);
#pragma unroll
            for (int r = 0; r < R1; ++r) S[(j + 16 * r) * 16 + c] = v[r];
        }
        __syncthreads();
        // stage 1, radix 16, span R1: butterfly j < R1 takes output j of every stage-0 butterfly r
        // (row r + 16 j), twiddled; its outputs are the spectrum at ky = j + R1 k
        if (j < R1) {
            float2 v[16];
#pragma unroll
            for (int r = 0; r < 16; ++r) v[r] = S[(r + 16 * j) * 16 + c];
#pragma unroll
            for (int r = 1; r < 16; ++r) v[r] = cmul(v[r], tw_f[(r - 1) * R1 + j]);
            dft<float, 16, false>(v);
            if (c < wv) {
#pragma unroll
                for (int k = 0; k < 16; ++k) out[(size_t)(j + R1 * k) * es] = v[k];
            }
        }
    } else {
        // stage 0, radix 16 (no twiddles): butterfly j < R1 on rows j + R1 r, outputs back in place
        if (j < R1) {
            float2 v[16];
#pragma unroll
            for (int r = 0; r < 16; ++r) v[r] = S[(j + R1 * r) * 16 + c];
            dft<float, 16, true>(v);
#pragma unroll
            for (int r = 0; r < 16; ++r) S[(j + R1 * r) * 16 + c] = v[r];
        }
        __syncthreads();
        // stage 1, radix R1, span 16: butterfly j < 16 takes output j of every stage-0 butterfly r
        // (row r + R1 j), conjugate-twiddled; its outputs are the line at y = j + 16 k
        {
            float2 v[R1];
#pragma unroll
            for (int r = 0; r < R1; ++r) v[r] = S[(r + R1 * j) * 16 + c];
#pragma unroll
            for (int r = 1; r < R1; ++r) v[r] = cmulc(v[r], tw_i[(r - 1) * 16 + j]);
            dft<float, R1, true>(v);
            if (c < wv) {
#pragma unroll
                for (int k = 0; k < R1; ++k) out[(size_t)(j + 16 * k) * es] = v[k];
            }
        }
    }
}

}  // namespace pat
