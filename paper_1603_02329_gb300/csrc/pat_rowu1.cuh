// pat_rowu1.cuh -- the momentum row kernels of 3-D grids (u update and its transpose) with one
// velocity component per CTA.
//
// The work of k_row2 with KIND = R2_FWD_U / R2_ADJ_U (Sec. II.A, the split u update with the PML;
// its exact transpose, Sec. III): inverse x-transform of the spectrum of D+-_xi, the pointwise
// update of u_xi, forward x-transform of its output.  Component xi's update reads only its own
// spectrum, b_xi, u_xi and its own PML factor, so a CTA takes R x-lines of one component
// (blockIdx.y = xi) with the same transform schedule, stages and arithmetic as k_row2 (the same
// helpers, one field instead of three): about a third of the shared memory and of the registers, so
// more CTAs per SM keep more lines in flight.  The checkpointed-gradient hooks are k_row2's.
#pragma once

#include "pat_row2.cuh"

namespace pat {

// shared memory: stage tables [2 nx] | A (np lines) | B (np lines, or the staged spectrum rows) |
// b_xi and u_xi rows [2][R][nx] | PML [nx + R]
template <typename T> struct RowU1Layout {
    size_t tab, lines, bsz, res, bytes;
};
template <typename T> __host__ __device__ RowU1Layout<T> rowu1_layout(int nx, int ldh, int R) {
    RowU1Layout<T> L;
    const int np = R / 2;
    L.tab = (size_t)2 * nx;
    L.lines = (size_t)np * nx + 2 * (size_t)p2_field_pad<T>();
    const size_t stg = (size_t)R * ldh;
    L.bsz = L.lines > stg ? L.lines : stg;
    L.res = (size_t)2 * R * nx;
    L.bytes = (L.tab + L.lines + L.bsz) * sizeof(cplx<T>) + (L.res + nx + ((R + 3) & ~3)) * sizeof(T);
    return L;
}

// LG: x-lines of 2^LG points; ADJ: the transpose (R2_ADJ_U).  grid (nlines / R, 3), 256 threads.
template <typename T, int LG, bool ADJ>
__global__ void __launch_bounds__(256) k_row_u1(DevPlan<T> P, int R, int flag) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int nx = 1 << LG;
    const int np = R >> 1, line0 = blockIdx.x * R, xi = blockIdx.y;
    const int lgnp = (np == 1) ? 0 : (np == 2 ? 1 : (np == 4 ? 2 : (np == 8 ? 3 : 4)));
    const RowU1Layout<T> Lo = rowu1_layout<T>(nx, P.ldh, R);
    cplx<T>* tab = reinterpret_cast<cplx<T>*>(smem_raw);
    cplx<T>* A = tab + Lo.tab;
    cplx<T>* B = A + Lo.lines;
    T* brow = reinterpret_cast<T*>(B + Lo.bsz);
    T* urow = brow + R * nx;
    T* pmlx = urow + R * nx;
    T* pmlr = pmlx + nx;
    const auto ax = P2Sel<LG>::make(P.fx.lgn);
    const T dt = P.dt;
    cplx<T>* const* spec = P.spec + xi;   // the one spectrum in and out

    // ---- prologue: tables and the medium (constants of the plan) ----
    stage16(tab, P.stw[0], (size_t)p2_tab_len(nx) * sizeof(cplx<T>));
    stage_rows(brow, P.b[xi], line0, R, nx);
    if (xi == 0) stage_elems(pmlx, P.au[0], nx);
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
        const int line = line0 + r;
        pmlr[r] = (xi == 0) ? (T)0 : P.au[xi][(xi == 1) ? line % P.ny : line / P.ny];
    }
    cp_commit();
    pdl_trigger();
    pdl_wait();

    // ---- state of the previous kernels: the spectrum rows and u_xi ----
    stage16(B, spec[0] + (size_t)line0 * P.ldh, (size_t)R * P.ldh * sizeof(cplx<T>));
    if (ADJ || !flag) stage_rows(urow, P.u[xi], line0, R, nx);
    cp_commit();
    cp_wait_all();
    __syncthreads();

    // ---- inverse x-transform of the spectrum ----
    p2_row_in<T>(A, B, 1, np, lgnp, ax, P.ldh);
    __syncthreads();
    cplx<T>* a = p2_mid<T, true>(A, B, ax, tab, np, lgnp);
    cplx<T>* bb = (a == A) ? B : A;

    auto pw = [&](int p, int j, int m, auto& z, auto& o) {
        constexpr int RR = sizeof(z[0]) / sizeof(z[0][0]);
        const int first = flag;
        r2_each<T, RR, 1, 1, 1, 1>(p, j, m, z, o, [&](int r, int x, const T* in, T* out) {
            const int t = r * nx + x;
            const size_t idx = (size_t)(line0 + r) * nx + x;
            const T bq = brow[t];
            const T au = (xi == 0) ? pmlx[x] : pmlr[r];
            if constexpr (!ADJ) {
                const T g = in[0];
                const T uo = first ? (T)0.5 * dt * bq * g : urow[t];
                const T un = au * (au * uo - dt * bq * g);
                P.u[xi][idx] = un;
                out[0] = un;
                if (P.hk_g[0]) P.hk_g[xi][idx] = g;
            } else {
                T ub = urow[t] + in[0];
                T g = -dt * bq * au * ub;
                const T ubn = ub;
                ub = au * au * ub;
                if (first) g += (T)0.5 * dt * bq * ub;
                P.u[xi][idx] = ub;
                out[0] = g;
                if (P.hk_gb[0]) {
                    const T gv = P.hk_gin[xi][idx];
                    T add = ubn * (-dt * au * gv);
                    if (first) add += ub * (T)0.5 * dt * gv;
                    P.hk_gb[xi][idx] += add;
                }
            }
        });
    };
    with_radix(ax.r0, [&](auto RC) { r2_fuse<T, decltype(RC)::value, 1, 1>(a, bb, tab, ax, np, lgnp, 1, 1, true, pw); });
    __syncthreads();
    cplx<T>* c = p2_mid<T, false>(bb, a, ax, tab, np, lgnp);
    p2_row_out<T>(c, spec, tab, ax, 1, np, lgnp, line0, P.ldh);
}

}  // namespace pat
