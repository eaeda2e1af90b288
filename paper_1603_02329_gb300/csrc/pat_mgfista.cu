// pat_mgfista.cu -- the host driver of the line-search multi-grid ISTA/FISTA (Alg. 3, Sec. V.E),
// plain ISTA (Alg. 1) and FISTA (Alg. 2), the power method for L_f (Sec. IV), and the coarse-level
// plan (Sec. V: half the points per axis, twice the spacing and the time step).
//
// Every vector operation runs in the library's kernels (pat_optim.cu) and every objective and
// gradient evaluation runs the forward / adjoint solves of the plans; the host only keeps the
// FP64 scalars (objective values, norms, step sizes, momentum) and takes the branch decisions,
// synchronising once per reduction.
#include <cmath>
#include <cstring>
#include <vector>

#include "pat_host.h"
#include "pat_optim.h"

namespace pat {

static pat_status fwd(pat_plan* p, const void* x, void* d, cudaStream_t s) { return pat_forward_plan(p, x, d, s); }
static pat_status adj(pat_plan* p, const void* r, void* g, cudaStream_t s) { return pat_adjoint(p, r, g, s); }

#define TRY(x)                       \
    do {                             \
        pat_status st_ = (x);        \
        if (st_ != PAT_OK) return st_; \
    } while (0)

template <typename T> struct Driver {
    static pat_status power(pat_plan* plan, const T* v0, int n_iter, double* L, cudaStream_t s) {
        const PlanBase* b = plan->impl;
        const long long N = b->info.N, M = (long long)b->info.Nt * b->info.Ns;
        T* buf = nullptr;
        cudaError_t e = cudaMallocAsync(&buf, (size_t)(2 * N + M) * sizeof(T), s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync (power method)");
        T* v = buf;
        T* w = buf + N;
        T* d = buf + 2 * N;
        double nv = 0.0;
        pat_status st = Ops<T>::reduce(HRED_DOT, nullptr, N, v0, v0, 0.0, &nv, s);
        if (st == PAT_OK) st = Ops<T>::lincomb(N, v, 1.0 / std::sqrt(nv), v0, 0.0, nullptr, 0.0, nullptr, nullptr, 0, s);
        double Lk = 0.0;
        for (int it = 0; it < n_iter && st == PAT_OK; ++it) {
            st = fwd(plan, v, d, s);
            if (st == PAT_OK) st = adj(plan, d, w, s);
            double n2 = 0.0;
            if (st == PAT_OK) st = Ops<T>::reduce(HRED_DOT, nullptr, N, w, w, 0.0, &n2, s);
            Lk = std::sqrt(n2);
            if (st == PAT_OK) st = Ops<T>::lincomb(N, v, 1.0 / Lk, w, 0.0, nullptr, 0.0, nullptr, nullptr, 0, s);
        }
        cudaFreeAsync(buf, s);
        *L = Lk;
        return st;
    }

    // Coarse-level FISTA / ISTA on phi = 1/2 ||H_c x - p_c||^2 + lam J_rho(x) + <v, x> with the
    // projection on {x >= lower} (Alg. 3 line 9; Sec. V.E).  x0 is x_{h-1,0}; result in xout.
    static pat_status coarse_solve(pat_plan* cp, const pat_grid* gc, const T* phat_c, const T* x0, const T* v,
                                   const T* lower, double L_c, double wc, const pat_fista_opts* o, T* xout,
                                   T* const* ws, T* const* wd, int* nfwd, int* nadj, cudaStream_t s) {
        const long long N = cp->impl->info.N, M = (long long)cp->impl->info.Nt * cp->impl->info.Ns;
        const double alpha = 1.0 / L_c, lam = o->lambda, rho = o->tv_rho;
        T* xp = ws[0];
        T* y = ws[1];
        T* g = ws[2];
        T* x = ws[3];
        T* Hxp = wd[0];
        T* Hy = wd[1];
        T* Hx = wd[2];
        T* r = wd[3];
        auto phi = [&](const T* xx, const T* Hxx, double* out) -> pat_status {
            double sq = 0.0, js = 0.0, vx = 0.0;
            TRY(Ops<T>::reduce(HRED_SQDIFF, nullptr, M, Hxx, phat_c, 0.0, &sq, s));
            TRY(Ops<T>::reduce(HRED_TVS, gc, N, xx, nullptr, rho, &js, s));
            TRY(Ops<T>::reduce(HRED_DOT, nullptr, N, v, xx, 0.0, &vx, s));
            *out = 0.5 * wc * sq + lam * js + vx;
            return PAT_OK;
        };
        TRY(Ops<T>::lincomb(N, xp, 1.0, x0, 0.0, nullptr, 0.0, nullptr, nullptr, 0, s));
        TRY(fwd(cp, xp, Hxp, s));
        ++*nfwd;
        TRY(Ops<T>::lincomb(N, y, 1.0, xp, 0.0, nullptr, 0.0, nullptr, nullptr, 0, s));
        TRY(Ops<T>::lincomb(M, Hy, 1.0, Hxp, 0.0, nullptr, 0.0, nullptr, nullptr, 0, s));
        double phi_prev = 0.0;
        TRY(phi(xp, Hxp, &phi_prev));
        double t = 1.0;
        for (int k = 1;; ++k) {
            // grad = w H_c^T (H_c y - p_c) + lam grad J_rho(y) + v
            TRY(Ops<T>::lincomb(M, r, 1.0, Hy, -1.0, phat_c, 0.0, nullptr, nullptr, 0, s));
            TRY(adj(cp, r, g, s));
            ++*nadj;
            TRY(Ops<T>::tv_smooth_grad(gc, y, rho, g, lam, wc, s));
            TRY(Ops<T>::lincomb(N, g, 1.0, g, 1.0, v, 0.0, nullptr, nullptr, 0, s));
            // x = max(y - alpha grad, lower)
            TRY(Ops<T>::lincomb(N, x, 1.0, y, -alpha, g, 0.0, nullptr, lower, 0, s));
            TRY(fwd(cp, x, Hx, s));
            ++*nfwd;
            double phi_x = 0.0;
            TRY(phi(x, Hx, &phi_x));
            double theta = 0.0;
            if (o->variant == 1) {
                const double tn = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t * t));
                theta = (t - 1.0) / tn;
                t = tn;
            }
            TRY(Ops<T>::lincomb(N, y, 1.0 + theta, x, -theta, xp, 0.0, nullptr, nullptr, 0, s));
            TRY(Ops<T>::lincomb(M, Hy, 1.0 + theta, Hx, -theta, Hxp, 0.0, nullptr, nullptr, 0, s));
            const double den = std::fmax(std::fmax(std::fabs(phi_prev), std::fabs(phi_x)), 1e-300);
            const double dec = (phi_prev - phi_x) / den;
            std::swap(xp, x);
            std::swap(Hxp, Hx);
            phi_prev = phi_x;
            if (dec < o->eps_c || k >= o->q_c) break;
        }
        return Ops<T>::lincomb(N, xout, 1.0, xp, 0.0, nullptr, 0.0, nullptr, nullptr, 0, s);
    }

    static pat_status run(pat_plan* fp, pat_plan* cp, const T* phat, const T* x0, const pat_fista_opts* o, T* xout,
                          pat_fista_report* rep, pat_iter_callback cb, void* ctx, cudaStream_t s) {
        const PlanBase* fb = fp->impl;
        const pat_grid gf = fb->in.grid;
        const long long N = fb->info.N, M = (long long)fb->info.Nt * fb->info.Ns;
        const int d = gf.ndim;
        pat_grid gc = gf;
        long long Nc = 0, Mc = 0;
        int Ntc = 0;
        if (cp) {
            for (int a = 0; a < d; ++a) gc.n[a] = gf.n[a] / 2;
            Nc = cp->impl->info.N;
            Ntc = cp->impl->info.Nt;
            Mc = (long long)Ntc * cp->impl->info.Ns;
        }
        // workspaces: fine image x 6, fine data x 4, coarse image x 10, coarse data x 5
        const size_t elems = (size_t)(6 * N + 4 * M + 10 * Nc + 5 * Mc);
        T* buf = nullptr;
        cudaError_t e = cudaMallocAsync(&buf, elems * sizeof(T), s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync (MG-FISTA)");
        T* p = buf;
        auto take = [&](long long n) {
            T* q = p;
            p += n;
            return q;
        };
        T* xp = take(N);
        T* x = take(N);
        T* y = take(N);
        T* g = take(N);
        T* z = take(N);
        T* ytil = take(N);
        T* Hxp = take(M);
        T* Hx = take(M);
        T* Hy = take(M);
        T* r = take(M);
        T* cimg[10];
        T* cdat[5];
        for (int k = 0; k < 10; ++k) cimg[k] = take(Nc);
        for (int k = 0; k < 5; ++k) cdat[k] = take(Mc);
        pat_status st = run_inner(fp, cp, gf, gc, N, M, Nc, Mc, Ntc, phat, x0, o, xout, rep, cb, ctx, s, xp, x, y, g,
                                  z, ytil, Hxp, Hx, Hy, r, cimg, cdat);
        cudaFreeAsync(buf, s);
        return st;
    }

    static pat_status run_inner(pat_plan* fp, pat_plan* cp, const pat_grid& gf, const pat_grid& gc, long long N,
                                long long M, long long Nc, long long Mc, int Ntc, const T* phat, const T* x0,
                                const pat_fista_opts* o, T* xout, pat_fista_report* rep, pat_iter_callback cb,
                                void* ctx, cudaStream_t s, T* xp, T* x, T* y, T* g, T* z, T* ytil, T* Hxp, T* Hx,
                                T* Hy, T* r, T* const* cimg, T* const* cdat) {
        const int d = gf.ndim;
        const double lam = o->lambda, rho = o->tv_rho;
        // weight of the coarse data term (O11): 2^(1-d) unless given
        const double wc = (o->coarse_weight > 0.0) ? o->coarse_weight : std::ldexp(1.0, 1 - gf.ndim);
        const double alpha = o->step_scale / o->L;
        const T* pex = static_cast<const T*>(o->p_exact);
        double nrm_exact = 0.0;
        if (pex) {
            TRY(Ops<T>::reduce(HRED_DOT, nullptr, N, pex, pex, 0.0, &nrm_exact, s));
            nrm_exact = std::sqrt(nrm_exact);
        }
        int nfwd = 0, nadj = 0, nrec = 0;
        auto F_of = [&](const T* xx, const T* Hxx, double* F, double* RES) -> pat_status {
            double sq = 0.0, tv = 0.0;
            TRY(Ops<T>::reduce(HRED_SQDIFF, nullptr, M, Hxx, phat, 0.0, &sq, s));
            TRY(Ops<T>::reduce(HRED_TV, &gf, N, xx, nullptr, 0.0, &tv, s));
            *F = 0.5 * sq + lam * tv;
            *RES = std::sqrt(sq);
            return PAT_OK;
        };
        auto norm = [&](const T* a, long long n, double* out) -> pat_status {
            double q = 0.0;
            TRY(Ops<T>::reduce(HRED_DOT, nullptr, n, a, a, 0.0, &q, s));
            *out = std::sqrt(q);
            return PAT_OK;
        };
        // coarse data: the fine record decimated in time (p_c^m = p^{2m})
        T* phat_c = cp ? cdat[4] : nullptr;
        if (cp) TRY(Ops<T>::decimate_rows(phat, phat_c, Ntc, cp->impl->info.Ns, s));

        TRY(Ops<T>::lincomb(N, xp, 1.0, x0, 0.0, nullptr, 0.0, nullptr, nullptr, 0, s));
        TRY(fwd(fp, xp, Hxp, s));
        ++nfwd;
        double F_prev = 0.0, RES0 = 0.0;
        TRY(F_of(xp, Hxp, &F_prev, &RES0));
        TRY(Ops<T>::lincomb(N, y, 1.0, xp, 0.0, nullptr, 0.0, nullptr, nullptr, 0, s));
        TRY(Ops<T>::lincomb(M, Hy, 1.0, Hxp, 0.0, nullptr, 0.0, nullptr, nullptr, 0, s));
        double t = 1.0;
        int K_d = 0, K_r = 0;
        bool have_ytil = false;
        double F_last = F_prev, RES_last = RES0, RE_last = NAN;
        int k = 0;
        for (k = 1; k <= o->max_iter; ++k) {
            // grad f(y_k) = H^T (H y_k - p_hat)   (Eq. (Six))
            TRY(Ops<T>::lincomb(M, r, 1.0, Hy, -1.0, phat, 0.0, nullptr, nullptr, 0, s));
            TRY(adj(fp, r, g, s));
            ++nadj;
            bool recursive = false;
            if (cp && o->recursion && k > 1) {
                // grad F_rho(y) (Eq. (Twentyone)) into z; R grad F_rho into cimg[8]
                TRY(Ops<T>::lincomb(N, z, 1.0, g, 0.0, nullptr, 0.0, nullptr, nullptr, 0, s));
                TRY(Ops<T>::tv_smooth_grad(&gf, y, rho, z, lam, 1.0, s));
                TRY(Ops<T>::restrict_(&gf, z, cimg[8], s));
                double nRg = 0.0, ngF = 0.0;
                TRY(norm(cimg[8], Nc, &nRg));
                TRY(norm(z, N, &ngF));
                const bool c1 = nRg > o->kappa * ngF;
                bool far = false;
                if (have_ytil) {
                    double ndiff = 0.0, nyt = 0.0;
                    TRY(Ops<T>::reduce(HRED_SQDIFF, nullptr, N, y, ytil, 0.0, &ndiff, s));
                    TRY(norm(ytil, N, &nyt));
                    far = std::sqrt(ndiff) > o->vartheta * nyt;
                }
                const bool c2 = far || K_r == 0 || K_d > o->q_d;
                recursive = c1 && c2;   // Eq. (conditions)
            }
            if (recursive) {
                K_d = 0;
                ++K_r;
                ++nrec;
                have_ytil = true;
                TRY(Ops<T>::lincomb(N, ytil, 1.0, y, 0.0, nullptr, 0.0, nullptr, nullptr, 0, s));
                T* xc0 = cimg[0];
                T* v = cimg[1];
                T* lower = cimg[2];
                T* gcb = cimg[3];
                T* xcs = cimg[9];
                // x_{h-1,0} = R y; v = R grad F_rho,h(y) - grad F_rho,h-1(x_{h-1,0})  (Eq. (Fourteen))
                TRY(Ops<T>::restrict_(&gf, y, xc0, s));
                TRY(fwd(cp, xc0, cdat[0], s));
                ++nfwd;
                TRY(Ops<T>::lincomb(Mc, cdat[1], 1.0, cdat[0], -1.0, phat_c, 0.0, nullptr, nullptr, 0, s));
                TRY(adj(cp, cdat[1], gcb, s));
                ++nadj;
                TRY(Ops<T>::tv_smooth_grad(&gc, xc0, rho, gcb, lam, wc, s));
                TRY(Ops<T>::lincomb(Nc, v, 1.0, cimg[8], -1.0, gcb, 0.0, nullptr, nullptr, 0, s));
                // restricted bound at y (Eq. (constraint))
                TRY(Ops<T>::coarse_bound(&gf, y, lower, cimg[4], s));
                const double L_c = wc * o->L_coarse + lam * 4.0 * d / rho;
                T* const ws[4] = {cimg[4], cimg[5], cimg[6], cimg[7]};
                T* const wd[4] = {cdat[0], cdat[1], cdat[2], cdat[3]};
                TRY(coarse_solve(cp, &gc, phat_c, xc0, v, lower, L_c, wc, o, xcs, ws, wd, &nfwd, &nadj, s));
                // x = y + P (x_{h-1,*} - x_{h-1,0})
                TRY(Ops<T>::lincomb(Nc, xcs, 1.0, xcs, -1.0, xc0, 0.0, nullptr, nullptr, 0, s));
                TRY(Ops<T>::lincomb(N, x, 1.0, y, 0.0, nullptr, 0.0, nullptr, nullptr, 0, s));
                TRY(Ops<T>::prolong(&gf, xcs, x, 1.0, 1.0, s));
            } else {
                ++K_d;
                // x = prox_{alpha g}(y - alpha grad f(y))   (Alg. 1 lines 3-4)
                TRY(Ops<T>::lincomb(N, z, 1.0, y, -alpha, g, 0.0, nullptr, nullptr, 0, s));
                TRY(Ops<T>::tv_prox(&gf, z, x, alpha * lam, o->n_tv, 1, s));
            }
            TRY(fwd(fp, x, Hx, s));
            ++nfwd;
            double F_x = 0.0, RES = 0.0;
            TRY(F_of(x, Hx, &F_x, &RES));
            double RE = NAN;
            if (pex) {
                double sq = 0.0;
                TRY(Ops<T>::reduce(HRED_SQDIFF, nullptr, N, x, pex, 0.0, &sq, s));
                RE = std::sqrt(sq) / nrm_exact;
            }
            if (cb) cb(ctx, k, recursive ? 1 : 0, F_x, RES, RE, nfwd, nadj);
            double theta = 0.0;
            if (o->variant == 1) {
                const double tn = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t * t));
                theta = (t - 1.0) / tn;
                t = tn;
            }
            TRY(Ops<T>::lincomb(N, y, 1.0 + theta, x, -theta, xp, 0.0, nullptr, nullptr, 0, s));
            TRY(Ops<T>::lincomb(M, Hy, 1.0 + theta, Hx, -theta, Hxp, 0.0, nullptr, nullptr, 0, s));
            const double dec = (F_prev - F_x) / std::fmax(F_prev, F_x);
            std::swap(xp, x);
            std::swap(Hxp, Hx);
            F_prev = F_x;
            F_last = F_x;
            RES_last = RES;
            RE_last = RE;
            if (dec < o->eps_d) break;
            if (o->target_re > 0.0 && pex && RE <= o->target_re) break;
        }
        TRY(Ops<T>::lincomb(N, xout, 1.0, xp, 0.0, nullptr, 0.0, nullptr, nullptr, 0, s));
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize (MG-FISTA)");
        if (rep) {
            rep->iters = std::min(k, o->max_iter);
            rep->recursive_iters = nrec;
            rep->fwd_solves = nfwd;
            rep->adj_solves = nadj;
            rep->F = F_last;
            rep->RES = RES_last;
            rep->RE = RE_last;
        }
        return PAT_OK;
    }
};

}  // namespace pat

using namespace pat;

extern "C" {

pat_status pat_power_iteration(pat_plan* plan, const void* v0, int n_iter, double* L, void* stream) {
    set_error("");
    if (!plan || !v0 || !L || n_iter < 1) {
        set_error("bad arguments");
        return PAT_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (plan->impl->info.precision == PAT_F32) return Driver<float>::power(plan, (const float*)v0, n_iter, L, s);
    return Driver<double>::power(plan, (const double*)v0, n_iter, L, s);
}

pat_status pat_plan_create_coarse(const pat_plan* fine, pat_plan** out) {
    set_error("");
    if (!fine || !out) {
        set_error("NULL argument");
        return PAT_EINVAL;
    }
    const PlanInputs& in = fine->impl->in;
    const pat_grid& g = in.grid;
    const int d = g.ndim;
    pat_grid gc = g;
    for (int a = 0; a < d; ++a) {
        if (g.n[a] % 4 != 0) {
            set_error("coarse level needs fine sizes divisible by 4 (even coarse sizes)");
            return PAT_EUNSUPPORTED;
        }
        gc.n[a] = g.n[a] / 2;
        gc.dx[a] = 2.0 * g.dx[a];
        gc.pml[a] = g.pml[a] / 2;
    }
    const int nx = g.n[0], ny = g.n[1], nz = (d == 3) ? g.n[2] : 1;
    const int cx = gc.n[0], cy = gc.n[1], cz = (d == 3) ? gc.n[2] : 1;
    const size_t Nc = (size_t)cx * cy * cz;
    std::vector<double> c(Nc), rho(Nc), a0(in.alpha0_is_scalar ? 1 : Nc);
    // medium decimated: coarse point i <- fine point 2 i
    for (int kz = 0; kz < cz; ++kz)
        for (int ky = 0; ky < cy; ++ky)
            for (int kx = 0; kx < cx; ++kx) {
                const size_t ic = ((size_t)kz * cy + ky) * cx + kx;
                const size_t jf = ((size_t)(2 * kz) * ny + 2 * ky) * nx + 2 * kx;
                c[ic] = in.c[jf];
                rho[ic] = in.rho[jf];
                if (!in.alpha0_is_scalar) a0[ic] = in.alpha0[jf];
            }
    (void)nz;
    if (in.alpha0_is_scalar) a0[0] = in.alpha0[0];
    // sensors at the same physical positions
    std::vector<double> pos;
    if (!in.pos.empty()) {
        pos = in.pos;
    } else {
        pos.resize((size_t)in.Ns * d);
        for (int j = 0; j < in.Ns; ++j) {
            long long idx = in.index[j];
            const int ix = (int)(idx % nx);
            idx /= nx;
            const int iy = (int)(idx % ny);
            const int iz = (int)(idx / ny);
            const int ci[3] = {ix, iy, iz};
            for (int a = 0; a < d; ++a) pos[(size_t)j * d + a] = (double)(ci[a] - g.n[a] / 2) * g.dx[a];
        }
    }
    // positions beyond the first / last coarse node are clamped onto it (as P clamps)
    for (int j = 0; j < in.Ns; ++j)
        for (int a = 0; a < d; ++a) {
            const double lo = (double)(0 - gc.n[a] / 2) * gc.dx[a];
            const double hi = (double)(gc.n[a] - 1 - gc.n[a] / 2) * gc.dx[a];
            double& v = pos[(size_t)j * d + a];
            v = std::fmin(std::fmax(v, lo), hi);
        }
    pat_sensors sc{in.Ns, pos.data(), nullptr};
    const int Ntc = (in.Nt + 1) / 2;
    return pat_plan_create(&gc, c.data(), rho.data(), a0.data(), in.alpha0_is_scalar, in.y, &sc, 2.0 * in.dt, Ntc,
                           in.prec, out);
}

pat_status pat_mg_fista(pat_plan* fine, pat_plan* coarse, const void* data, const void* x0,
                        const pat_fista_opts* opts, void* x_out, pat_fista_report* report, pat_iter_callback cb,
                        void* cb_ctx, void* stream) {
    set_error("");
    if (!fine || !data || !x0 || !opts || !x_out) {
        set_error("NULL argument");
        return PAT_EINVAL;
    }
    if (!(opts->L > 0.0) || (coarse && opts->recursion && !(opts->L_coarse > 0.0)) || opts->max_iter < 0 ||
        !(opts->tv_rho > 0.0)) {
        set_error("bad options (L, L_coarse, tv_rho must be > 0)");
        return PAT_EINVAL;
    }
    if (coarse && (coarse->impl->info.precision != fine->impl->info.precision ||
                   coarse->impl->info.Ns != fine->impl->info.Ns ||
                   coarse->impl->info.Nt != (fine->impl->info.Nt + 1) / 2)) {
        set_error("coarse plan does not match the fine plan (use pat_plan_create_coarse)");
        return PAT_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (fine->impl->info.precision == PAT_F32)
        return Driver<float>::run(fine, coarse, (const float*)data, (const float*)x0, opts, (float*)x_out, report, cb,
                                  cb_ctx, s);
    return Driver<double>::run(fine, coarse, (const double*)data, (const double*)x0, opts, (double*)x_out, report, cb,
                               cb_ctx, s);
}

}  // extern "C"
