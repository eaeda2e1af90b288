// pat_row2.cuh -- row kernels of the per-phase path for power-of-two x-lines.
//
// The same work as k_fwd_u, k_fwd_rho, k_fwd_p, k_adj_rho, k_adj_u, k_adj_p (pat_kernels.cuh):
// the x-transforms of a step, fused with its pointwise physics (Sec. II.A; the exact transpose in
// the adjoint, Sec. III), for R consecutive x-lines per CTA.  The transform follows the fixed
// power-of-two Stockham schedule of the persistent kernel (pat_persist2.cuh):
//   * the spectra and the state rows are staged with cp.async into shared memory;
//   * inverse stage 0 does the C2R packing of two real lines on the loaded values;
//   * the last inverse stage, the pointwise physics and the first forward stage run in registers on
//     the same elements (one thread holds every field of its elements);
//   * the last forward stage holds X[k] and X[n-k] together, unpacks in registers and stores the
//     half spectra directly.
// Updated state goes straight from registers to global memory.  Sensor sampling reads the new
// pressure from a shared buffer after the pointwise step; the adjoint injects M^T h through the
// same buffer before it.  Checkpointed-gradient hooks (q^n = dp/dc0^2, g_c2 += p_bar q) are those of
// the generic kernels.
#pragma once

#include "pat_persist2.cuh"

namespace pat {

// Last inverse x-stage (radix R) of FI <= FIM fields, the pointwise step pw(p, j, m, z, o) with every
// field of butterfly (p, j) in one thread, and -- when `fwd` -- forward x-stage 0 of FO <= FOM outputs.
template <typename T, int R, int FIM, int FOM, class AX, class PW>
__device__ __forceinline__ void r2_fuse(const cplx<T>* src, cplx<T>* dst, const cplx<T>* tab, const AX& ax,
                                        int np, int lgnp, int FI, int FO, bool fwd, PW&& pw) {
    constexpr bool CM = P2IsC<AX>::value;
    const int n = ax.n, lgm = ax.lg - Lg2<R>::v, m = 1 << lgm;
    const cplx<T>* twl = tab + p2_off_i(ax, ax.nst - 1);
    for (int t = threadIdx.x; t < (np << lgm); t += blockDim.x) {
        const int p = t >> lgm, j = t & (m - 1);
        cplx<T> z[FIM][R], o[FOM][R];
#pragma unroll
        for (int f = 0; f < FIM; ++f) {
            if (f < FI) {
                p2_load<T, R, true, CM>(z[f], src + lbase<T>(f * np + p, n, lgnp), j, m, m, twl);
                dft<T, R, true>(z[f]);
            }
        }
        pw(p, j, m, z, o);
        if (fwd) {
#pragma unroll
            for (int g = 0; g < FOM; ++g) {
                if (g < FO) {
                    dft<T, R, false>(o[g]);
                    p2_store<T, R, CM>(dst + lbase<T>(g * np + p, n, lgnp), j, 1, o[g]);
                }
            }
        }
    }
}

// elementwise loop of a pointwise step: f(row, x, in[FI], out[FO]) over the 2R real elements of
// butterfly (p, j) (rows 2p, 2p+1; x = j + r m)
template <typename T, int R, int FIM, int FOM, int FI, int FO, class F>
__device__ __forceinline__ void r2_each(int p, int j, int m, const cplx<T> (&z)[FIM][R], cplx<T> (&o)[FOM][R],
                                        F&& f) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            T in[FIM > 0 ? FIM : 1], out[FOM] = {};
#pragma unroll
            for (int q = 0; q < FI; ++q) in[q] = h ? z[q][r].y : z[q][r].x;
            f(2 * p + h, j + r * m, in, out);
#pragma unroll
            for (int g = 0; g < FO; ++g) {
                if (h) o[g][r].y = out[g];
                else o[g][r].x = out[g];
            }
        }
    }
}

// LG > 0: compiled for x-lines of 2^LG points (the launcher checks the plan); 0: any power of two
template <typename T, int D, int KIND, int LG = 0>
__global__ void __launch_bounds__(256) k_row2(DevPlan<T> P, int R, int flag, T* data_row, const T* h_row, T* qrow,
                                              T* gc2, const T* p0c) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nx = LG ? (1 << LG) : P.nx, np = R >> 1, line0 = blockIdx.x * R;
    const int lgnp = (np == 1) ? 0 : (np == 2 ? 1 : (np == 4 ? 2 : (np == 8 ? 3 : 4)));
    const Row2Layout<T> Lo = row2_layout<T>(D, nx, P.ldh, R);
    cplx<T>* tab = reinterpret_cast<cplx<T>*>(smem_raw);
    cplx<T>* A = tab + Lo.tab;
    cplx<T>* B = A + Lo.lines;
    cplx<T>* gb = B + Lo.bsz;
    T* res = reinterpret_cast<T*>(gb + Lo.gb);
    T* pmlx = res + Lo.res;
    T* pmlr = pmlx + nx;
    auto row = [&](int k) { return res + k * R * nx; };
    const auto ax = P2Sel<LG>::make(P.fx.lgn);
    const T dt = P.dt;
    const bool lossy = P.lossy != 0;

    // ---- prologue: tables and the medium (constants of the plan) ----
    stage16(tab, P.stw[0], (size_t)p2_tab_len(nx) * sizeof(cplx<T>));
    int FI = D, FO = D;
    bool fwd = true, gath = false, scat = false;
    const T* const* pml_tab = P.a;
    switch (KIND) {
        case R2_FWD_U:
            pml_tab = P.au;
#pragma unroll
            for (int xi = 0; xi < D; ++xi) stage_rows(row(xi), P.b[xi], line0, R, nx);
            break;
        case R2_FWD_RHO:
            stage_rows(row(0), P.rho0, line0, R, nx);
            if (!lossy) stage_rows(row(1), P.c2, line0, R, nx);
            FO = lossy ? 2 : 1;
            fwd = lossy || !flag;
            gath = !lossy && !P.atd;
            scat = P.atd != 0;   // adjoint-then-discretize: the source M^T atd_row
            break;
        case R2_FWD_P:
            stage_rows(row(0), P.c2, line0, R, nx);
            stage_rows(row(1), P.c2tau, line0, R, nx);
            stage_rows(row(2), P.c2eta, line0, R, nx);
            FI = 2;
            FO = 1;
            fwd = !flag;
            gath = true;
            break;
        case R2_ADJ_RHO:
            stage_rows(row(0), P.c2, line0, R, nx);
            stage_rows(row(1), P.rho0, line0, R, nx);
            FI = 2;
            break;
        case R2_ADJ_U:
            pml_tab = P.au;
#pragma unroll
            for (int xi = 0; xi < D; ++xi) stage_rows(row(xi), P.b[xi], line0, R, nx);
            break;
        default:   // R2_ADJ_P
            if (lossy && !flag) {
                stage_rows(row(0), P.c2tau, line0, R, nx);
                stage_rows(row(1), P.c2eta, line0, R, nx);
            } else {
                stage_rows(row(0), P.c2, line0, R, nx);
                stage_rows(row(1), P.rho0, line0, R, nx);
            }
            FI = 1;
            FO = lossy ? 2 : D;
            fwd = !flag;
            scat = true;
            break;
    }
    stage_elems(pmlx, pml_tab[0], nx);
    for (int t = threadIdx.x; t < (D - 1) * R; t += blockDim.x) {
        const int a = 1 + t / R, r = t - (a - 1) * R;
        const int line = line0 + r;
        pmlr[t] = pml_tab[a][(a == 1) ? line % P.ny : line / P.ny];
    }
    cp_commit();
    // adjoint: M^T h^n into the zeroed buffer gb (the residual record is read-only during the
    // adjoint solve; segments are distinct points), read back by the pointwise step
    const DevSensors<T>& S = P.sens;
    if (scat) {
        const T* hr = (KIND == R2_FWD_RHO) ? P.atd_row : h_row;
        for (int t = threadIdx.x; t < np * nx; t += blockDim.x) gb[t] = mkc<T>(0, 0);
        __syncthreads();
        const int s0 = S.s_lineptr[line0], s1 = S.s_lineptr[line0 + R];
        for (int q = s0 + threadIdx.x; q < s1; q += blockDim.x) {
            T acc = 0;
            for (int e = S.s_seg_e0[q]; e < S.s_seg_e0[q + 1]; ++e) acc += S.s_ent_w[e] * hr[S.s_ent_sensor[e]];
            const int pos = (S.s_seg_line[q] - line0) * nx + S.s_seg_x[q];
            const int r = pos / nx, x = pos - r * nx;
            slot(gb, r, x, nx) += acc;
        }
    }
    pdl_trigger();
    pdl_wait();

    // ---- state of the previous kernels: spectra and state rows ----
    for (int f = 0; f < FI; ++f)
        stage16(B + (size_t)f * R * P.ldh, P.spec[f] + (size_t)line0 * P.ldh, (size_t)R * P.ldh * sizeof(cplx<T>));
    switch (KIND) {
        case R2_FWD_U:
            if (!flag) {
#pragma unroll
                for (int xi = 0; xi < D; ++xi) stage_rows(row(D + xi), P.u[xi], line0, R, nx);
            }
            break;
        case R2_FWD_RHO:
#pragma unroll
            for (int xi = 0; xi < D; ++xi) stage_rows(row(2 + xi), P.rh[xi], line0, R, nx);
            break;
        case R2_FWD_P:
            stage_rows(row(3), P.rsum, line0, R, nx);
            break;
        case R2_ADJ_RHO:
            stage_rows(row(2), P.pbar, line0, R, nx);
#pragma unroll
            for (int xi = 0; xi < D; ++xi) stage_rows(row(3 + xi), P.rh[xi], line0, R, nx);
            break;
        case R2_ADJ_U:
#pragma unroll
            for (int xi = 0; xi < D; ++xi) stage_rows(row(D + xi), P.u[xi], line0, R, nx);
            break;
        default:
            if (!(lossy && !flag)) {
#pragma unroll
                for (int xi = 0; xi < D; ++xi) stage_rows(row(2 + xi), P.rh[xi], line0, R, nx);
            }
            break;
    }
    cp_commit();
    cp_wait_all();
    __syncthreads();

    // ---- inverse x-transform of the FI spectra ----
    p2_row_in<T>(A, B, FI, np, lgnp, ax, P.ldh);
    __syncthreads();
    cplx<T>* a = p2_mid<T, true>(A, B, ax, tab, FI * np, lgnp);
    cplx<T>* bb = (a == A) ? B : A;

    auto pml = [&](int xi, int r, int x) { return xi == 0 ? pmlx[x] : pmlr[(xi - 1) * R + r]; };
    auto gidx = [&](int r, int x) { return (size_t)(line0 + r) * nx + x; };
    constexpr int FIM = D, FOM = D;
    auto pw = [&](int p, int j, int m, auto& z, auto& o) {
        constexpr int RR = sizeof(z[0]) / sizeof(z[0][0]);
        const int first = flag;
        switch (KIND) {
            case R2_FWD_U:
                r2_each<T, RR, FIM, FOM, D, D>(p, j, m, z, o, [&](int r, int x, const T* in, T* out) {
                    const int t = r * nx + x;
                    const size_t idx = gidx(r, x);
#pragma unroll
                    for (int xi = 0; xi < D; ++xi) {
                        const T g = in[xi];
                        const T bq = row(xi)[t];
                        const T au = pml(xi, r, x);
                        const T uo = first ? (T)0.5 * dt * bq * g : row(D + xi)[t];
                        const T un = au * (au * uo - dt * bq * g);
                        P.u[xi][idx] = un;
                        out[xi] = un;
                        if (P.hk_g[0]) P.hk_g[xi][idx] = g;
                    }
                });
                break;
            case R2_FWD_RHO:
                r2_each<T, RR, FIM, FOM, D, 2>(p, j, m, z, o, [&](int r, int x, const T* in, T* out) {
                    const int t = r * nx + x;
                    const size_t idx = gidx(r, x);
                    const T rho0 = row(0)[t];
                    const T src = P.atd ? slot(gb, r, x, nx) : (T)0;
                    const int trj = P.tr_node ? P.tr_node[idx] : -1;
                    T rs = 0, es = 0;
#pragma unroll
                    for (int xi = 0; xi < D; ++xi) {
                        const T e = in[xi];
                        const T aa = pml(xi, r, x);
                        const T rh = P.atd ? aa * (aa * row(2 + xi)[t] - dt * rho0 * e + dt * rho0 * src / T(D))
                                           : aa * (aa * row(2 + xi)[t] - dt * rho0 * e);
                        P.rh[xi][idx] = (trj >= 0) ? P.tr_row[trj] / (T(D) * P.c2[idx]) : rh;
                        rs += rh;
                        es += e;
                        if (P.hk_e[0]) P.hk_e[xi][idx] = e;
                    }
                    if (lossy) {
                        P.rsum[idx] = rs;
                        if (P.atd) {
                            out[0] = P.c2tau[idx] * (src - es);
                            out[1] = P.c2eta[idx] * rs / rho0;
                        } else {
                            out[0] = rho0 * es;
                            out[1] = rs;
                        }
                    } else {
                        T pv = row(1)[t] * rs;
                        if (trj >= 0) pv = P.tr_row[trj];
                        if (P.tr_img && flag) P.tr_img[idx] = pv;
                        slot(gb, r, x, nx) = pv;
                        if (qrow) qrow[idx] = rs;   // d p / d c0^2 (lossless)
                        out[0] = pv;
                    }
                });
                break;
            case R2_FWD_P:
                r2_each<T, RR, FIM, FOM, 2, 1>(p, j, m, z, o, [&](int r, int x, const T* in, T* out) {
                    const int t = r * nx + x;
                    const T c2 = row(0)[t], rs = row(3)[t];
                    const size_t idx = gidx(r, x);
                    T pv;
                    if (P.atd) {
                        const T rho0 = P.rho0[idx];
                        pv = c2 * rs - rho0 * in[0] - rho0 * in[1];
                    } else {
                        pv = c2 * rs + row(1)[t] * in[0] - row(2)[t] * in[1];
                    }
                    if (P.tr_node) {
                        const int trj = P.tr_node[idx];
                        if (trj >= 0) pv = P.tr_row[trj];
                    }
                    if (P.tr_img && flag) P.tr_img[idx] = pv;
                    slot(gb, r, x, nx) = pv;
                    if (qrow)   // d p / d c0^2 with tau, eta following c0 (Eq. (Twelve))
                        qrow[gidx(r, x)] =
                            rs + ((P.phb + (T)1) * row(1)[t] * in[0] - (P.pha + (T)2) * row(2)[t] * in[1]) / c2;
                    out[0] = pv;
                });
                break;
            case R2_ADJ_RHO:
                r2_each<T, RR, FIM, FOM, 2, D>(p, j, m, z, o, [&](int r, int x, const T* in, T* out) {
                    const int t = r * nx + x;
                    const size_t idx = gidx(r, x);
                    const T ddbar = in[0];
                    const T rbar = row(0)[t] * row(2)[t] - in[1];
                    const T rho0 = row(1)[t];
                    T gr = 0;
#pragma unroll
                    for (int xi = 0; xi < D; ++xi) {
                        const T aa = pml(xi, r, x);
                        const T rb = row(3 + xi)[t] + rbar;
                        out[xi] = rho0 * ddbar - dt * rho0 * aa * rb;
                        P.rh[xi][idx] = aa * aa * rb;
                        if (P.hk_grho) gr += P.hk_ein[xi][idx] * (ddbar - dt * aa * rb);
                    }
                    if (P.hk_grho) P.hk_grho[idx] += gr;
                });
                break;
            case R2_ADJ_U:
                r2_each<T, RR, FIM, FOM, D, D>(p, j, m, z, o, [&](int r, int x, const T* in, T* out) {
                    const int t = r * nx + x;
                    const size_t idx = gidx(r, x);
#pragma unroll
                    for (int xi = 0; xi < D; ++xi) {
                        const T bq = row(xi)[t];
                        const T au = pml(xi, r, x);
                        T ub = row(D + xi)[t] + in[xi];
                        T g = -dt * bq * au * ub;
                        const T ubn = ub;
                        ub = au * au * ub;
                        if (first) g += (T)0.5 * dt * bq * ub;
                        P.u[xi][idx] = ub;
                        out[xi] = g;
                        if (P.hk_gb[0]) {
                            const T gv = P.hk_gin[xi][idx];
                            T add = ubn * (-dt * au * gv);
                            if (first) add += ub * (T)0.5 * dt * gv;
                            P.hk_gb[xi][idx] += add;
                        }
                    }
                });
                break;
            default:   // R2_ADJ_P: p_bar = transpose of g = D+ p (spectrum 0) + M^T h, then the tail
                r2_each<T, RR, FIM, FOM, 1, D>(p, j, m, z, o, [&](int r, int x, const T* in, T* out) {
                    const int t = r * nx + x;
                    const size_t idx = gidx(r, x);
                    const T pv = in[0] + slot(gb, r, x, nx);
                    if (first) {   // final level: the transpose of the initial state
                        T s = 0;
#pragma unroll
                        for (int xi = 0; xi < D; ++xi) s += row(2 + xi)[t];
                        const T c2 = row(0)[t];
                        P.img[idx] = pv + s / (T(D) * c2);
                        if (gc2) gc2[idx] -= s * p0c[idx] / (T(D) * c2 * c2);
                        return;
                    }
                    if (gc2) gc2[idx] += pv * qrow[idx];
                    if (lossy) {
                        P.pbar[idx] = pv;
                        out[0] = row(0)[t] * pv;
                        out[1] = row(1)[t] * pv;
                    } else {
                        const T rbar = row(0)[t] * pv;
                        const T rho0 = row(1)[t];
                        T gr = 0;
#pragma unroll
                        for (int xi = 0; xi < D; ++xi) {
                            const T aa = pml(xi, r, x);
                            const T rb = row(2 + xi)[t] + rbar;
                            out[xi] = -dt * rho0 * aa * rb;
                            P.rh[xi][idx] = aa * aa * rb;
                            if (P.hk_grho) gr += P.hk_ein[xi][idx] * (-dt * aa * rb);
                        }
                        if (P.hk_grho) P.hk_grho[idx] += gr;
                    }
                });
                break;
        }
    };
    with_radix(ax.r0, [&](auto RC) {
        r2_fuse<T, decltype(RC)::value, FIM, FOM>(a, bb, tab, ax, np, lgnp, FI, FO, fwd, pw);
    });
    __syncthreads();
    if (gath) {
        // s^{n+1}_j += this CTA's part of sensor j (one atomic add per (line, sensor) segment)
        const int s0 = S.g_lineptr[line0], s1 = S.g_lineptr[line0 + R];
        for (int q = s0 + threadIdx.x; q < s1; q += blockDim.x) {
            const int j = S.g_seg_sensor[q];
            const int pos = (S.g_seg_line[q] - line0) * nx + S.g_seg_x0[q];
            const T w0 = S.g_seg_w0[q], w1 = S.g_seg_w1[q];
            const int r = pos / nx, x = pos - r * nx;
            T acc = w0 * slot(gb, r, x, nx);
            if (w1 != (T)0) acc += w1 * slot(gb, r, x + 1, nx);
            atomicAdd(&data_row[j], acc);
        }
    }
    if (!fwd) return;
    cplx<T>* c = p2_mid<T, false>(bb, a, ax, tab, FO * np, lgnp);
    p2_row_out<T>(c, P.spec, tab, ax, FO, np, lgnp, line0, P.ldh);
}

}  // namespace pat
