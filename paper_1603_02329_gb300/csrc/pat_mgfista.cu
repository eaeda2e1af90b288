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
#include <string>
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

    // One coarse level of the hierarchy (levels 1 .. nl - 1 below the fine level 0): its plan, grid
    // and sizes, L(H^T H), the weight w of its data term (O11 per level step) and its work arrays.
    struct Lev {
        pat_plan* plan = nullptr;
        pat_grid grid{};
        long long N = 0, M = 0;
        int Nt = 0, Ns = 0;
        double Ld = 0.0, w = 1.0;
        // images: start x_{l,0}, coherence term v_l, bound b_l, gradient of the level's own data and
        // TV terms at x_{l,0}, result x_{l,*}, the FISTA iterates, y~, the restricted gradient of
        // the level above, scratch of the restricted bound
        T *x0, *v, *lower, *gcb, *xs, *xp, *y, *gr, *x, *ytil, *rg, *tmp;
        // data: p_hat_l (decimated in time), H x_prev, H y, H x, residual
        T *phat, *Hxp, *Hy, *Hx, *r;
    };
    struct Count {
        int nfwd = 0, nadj = 0;
    };

    // Level-l FISTA / ISTA on phi_l = w_l/2 ||H_l x - p_l||^2 + lam J_rho(x) + <v_l, x> with the
    // projection on {x >= b_l} (Alg. 3 line 9; Sec. V.E), from x_{l,0} into x_{l,*}.  When a level
    // l + 1 exists, an iteration k > 1 takes a recursive direction under the test of Sec. V.D
    // applied to phi_l, with the bound restricted from b_l (the multi-level reading of the oracle,
    // O12); with two levels this is the coarse solve of Alg. 3 exactly.
    static pat_status level_solve(Lev* lv, int nl, int l, const pat_fista_opts* o, Count* cnt, cudaStream_t s) {
        Lev& L = lv[l];
        const long long N = L.N, M = L.M;
        const int d = L.grid.ndim;
        const double lam = o->lambda, rho = o->tv_rho;
        const double L_c = L.w * L.Ld + lam * 4.0 * d / rho;
        const double alpha = 1.0 / L_c;
        T* xp = L.xp;
        T* x = L.x;
        T* Hxp = L.Hxp;
        T* Hx = L.Hx;
        T* y = L.y;
        T* g = L.gr;
        T* Hy = L.Hy;
        T* r = L.r;
        auto phi = [&](const T* xx, const T* Hxx, double* out) -> pat_status {
            double sq = 0.0, js = 0.0, vx = 0.0;
            TRY(Ops<T>::reduce(HRED_SQDIFF, nullptr, M, Hxx, L.phat, 0.0, &sq, s));
            TRY(Ops<T>::reduce(HRED_TVS, &L.grid, N, xx, nullptr, rho, &js, s));
            TRY(Ops<T>::reduce(HRED_DOT, nullptr, N, L.v, xx, 0.0, &vx, s));
            *out = 0.5 * L.w * sq + lam * js + vx;
            return PAT_OK;
        };
        auto norm = [&](const T* a, long long n, double* out) -> pat_status {
            double q = 0.0;
            TRY(Ops<T>::reduce(HRED_DOT, nullptr, n, a, a, 0.0, &q, s));
            *out = std::sqrt(q);
            return PAT_OK;
        };
        TRY(Ops<T>::lincomb(N, xp, 1.0, L.x0, 0.0, nullptr, 0.0, nullptr, nullptr, 0, s));
        TRY(fwd(L.plan, xp, Hxp, s));
        ++cnt->nfwd;
        TRY(Ops<T>::lincomb(N, y, 1.0, xp, 0.0, nullptr, 0.0, nullptr, nullptr, 0, s));
        TRY(Ops<T>::lincomb(M, Hy, 1.0, Hxp, 0.0, nullptr, 0.0, nullptr, nullptr, 0, s));
        double phi_prev = 0.0;
        TRY(phi(xp, Hxp, &phi_prev));
        double t = 1.0;
        int K_d = 0, K_r = 0;
        bool have_ytil = false;
        for (int k = 1;; ++k) {
            // grad phi_l(y) = w H^T (H y - p) + lam grad J_rho(y) + v
            TRY(Ops<T>::lincomb(M, r, 1.0, Hy, -1.0, L.phat, 0.0, nullptr, nullptr, 0, s));
            TRY(adj(L.plan, r, g, s));
            ++cnt->nadj;
            TRY(Ops<T>::tv_smooth_grad(&L.grid, y, rho, g, lam, L.w, s));
            TRY(Ops<T>::lincomb(N, g, 1.0, g, 1.0, L.v, 0.0, nullptr, nullptr, 0, s));
            bool recursive = false;
            if (l + 1 < nl && o->recursion && k > 1) {
                Lev& C = lv[l + 1];
                TRY(Ops<T>::restrict_(&L.grid, g, C.rg, s));
                double nRg = 0.0, ng = 0.0;
                TRY(norm(C.rg, C.N, &nRg));
                TRY(norm(g, N, &ng));
                bool far = false;
                if (have_ytil) {
                    double ndiff = 0.0, nyt = 0.0;
                    TRY(Ops<T>::reduce(HRED_SQDIFF, nullptr, N, y, L.ytil, 0.0, &ndiff, s));
                    TRY(norm(L.ytil, N, &nyt));
                    far = std::sqrt(ndiff) > o->vartheta * nyt;
                }
                recursive = (nRg > o->kappa * ng) && (far || K_r == 0 || K_d > o->q_d);
            }
            if (recursive) {
                K_d = 0;
                ++K_r;
                have_ytil = true;
                TRY(Ops<T>::lincomb(N, L.ytil, 1.0, y, 0.0, nullptr, 0.0, nullptr, nullptr, 0, s));
                TRY(coarse_step(lv, nl, l + 1, &L.grid, y, L.lower, o, cnt, s));
                TRY(Ops<T>::lincomb(N, x, 1.0, y, 0.0, nullptr, 0.0, nullptr, nullptr, 0, s));
                TRY(Ops<T>::prolong(&L.grid, lv[l + 1].xs, x, 1.0, 1.0, s));
            } else {
                ++K_d;
                // x = max(y - alpha grad, lower)
                TRY(Ops<T>::lincomb(N, x, 1.0, y, -alpha, g, 0.0, nullptr, L.lower, 0, s));
            }
            TRY(fwd(L.plan, x, Hx, s));
            ++cnt->nfwd;
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
        return Ops<T>::lincomb(N, L.xs, 1.0, xp, 0.0, nullptr, 0.0, nullptr, nullptr, 0, s);
    }

    // Recursive search direction from the level above level c (Alg. 3 lines 4-10): with C.rg =
    // R grad of the level above at y, set x_{c,0} = R y, v_c = R grad - grad(w_c/2 ||H_c x - p_c||^2
    // + lam J_rho)(x_{c,0}) (Eq. (Fourteen)), the bound restricted at y (Eq. (constraint); from
    // b_above when the level above has a bound, O12), solve level c, and leave x_{c,*} - x_{c,0} in
    // C.xs for the caller to prolong.
    static pat_status coarse_step(Lev* lv, int nl, int c, const pat_grid* gabove, const T* y, const T* b_above,
                                  const pat_fista_opts* o, Count* cnt, cudaStream_t s) {
        Lev& C = lv[c];
        const double lam = o->lambda, rho = o->tv_rho;
        TRY(Ops<T>::restrict_(gabove, y, C.x0, s));
        TRY(fwd(C.plan, C.x0, C.Hxp, s));
        ++cnt->nfwd;
        TRY(Ops<T>::lincomb(C.M, C.r, 1.0, C.Hxp, -1.0, C.phat, 0.0, nullptr, nullptr, 0, s));
        TRY(adj(C.plan, C.r, C.gcb, s));
        ++cnt->nadj;
        TRY(Ops<T>::tv_smooth_grad(&C.grid, C.x0, rho, C.gcb, lam, C.w, s));
        TRY(Ops<T>::lincomb(C.N, C.v, 1.0, C.rg, -1.0, C.gcb, 0.0, nullptr, nullptr, 0, s));
        TRY(Ops<T>::coarse_bound(gabove, y, C.lower, C.tmp, s, b_above));
        TRY(level_solve(lv, nl, c, o, cnt, s));
        return Ops<T>::lincomb(C.N, C.xs, 1.0, C.xs, -1.0, C.x0, 0.0, nullptr, nullptr, 0, s);
    }

    // plans[0] is the fine level, plans[l] the level below plans[l - 1] (pat_plan_create_coarse);
    // Ls[l] = L(H_l^T H_l) from the power method
    static pat_status run(pat_plan* const* plans, int nl, const double* Ls, const T* phat, const T* x0,
                          const pat_fista_opts* o, T* xout, pat_fista_report* rep, pat_iter_callback cb, void* ctx,
                          cudaStream_t s) {
        const PlanBase* fb = plans[0]->impl;
        const pat_grid gf = fb->in.grid;
        const long long N = fb->info.N, M = (long long)fb->info.Nt * fb->info.Ns;
        // weight of the coarse data term per level step (O11): 2^(1-d) unless given
        const double wc = (o->coarse_weight > 0.0) ? o->coarse_weight : std::ldexp(1.0, 1 - gf.ndim);
        std::vector<Lev> lv((size_t)nl);
        // workspaces: fine image x 6, fine data x 4; per coarse level image x 12, data x 5
        size_t elems = (size_t)(6 * N + 4 * M);
        for (int l = 1; l < nl; ++l) {
            Lev& L = lv[l];
            L.plan = plans[l];
            L.grid = plans[l]->impl->in.grid;
            L.N = plans[l]->impl->info.N;
            L.Nt = plans[l]->impl->info.Nt;
            L.Ns = plans[l]->impl->info.Ns;
            L.M = (long long)L.Nt * L.Ns;
            L.Ld = Ls[l];
            L.w = (l == 1) ? wc : lv[l - 1].w * wc;
            elems += (size_t)(12 * L.N + 5 * L.M);
        }
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
        for (int l = 1; l < nl; ++l) {
            Lev& L = lv[l];
            T** im[12] = {&L.x0, &L.v, &L.lower, &L.gcb, &L.xs, &L.xp, &L.y, &L.gr, &L.x, &L.ytil, &L.rg, &L.tmp};
            for (T** q : im) *q = take(L.N);
            T** da[5] = {&L.phat, &L.Hxp, &L.Hy, &L.Hx, &L.r};
            for (T** q : da) *q = take(L.M);
        }
        pat_status st = PAT_OK;
        // data of each coarse level: the record of the level above decimated in time (p_c^m = p^{2m})
        for (int l = 1; l < nl && st == PAT_OK; ++l)
            st = Ops<T>::decimate_rows(l == 1 ? phat : lv[l - 1].phat, lv[l].phat, lv[l].Nt, lv[l].Ns, s);
        if (st == PAT_OK)
            st = run_inner(plans[0], gf, N, M, lv.data(), nl, phat, x0, o, xout, rep, cb, ctx, s, xp, x, y, g, z,
                           ytil, Hxp, Hx, Hy, r);
        cudaFreeAsync(buf, s);
        return st;
    }

    static pat_status run_inner(pat_plan* fp, const pat_grid& gf, long long N, long long M, Lev* lv, int nl,
                                const T* phat, const T* x0, const pat_fista_opts* o, T* xout, pat_fista_report* rep,
                                pat_iter_callback cb, void* ctx, cudaStream_t s, T* xp, T* x, T* y, T* g, T* z,
                                T* ytil, T* Hxp, T* Hx, T* Hy, T* r) {
        const double lam = o->lambda, rho = o->tv_rho;
        const double alpha = o->step_scale / o->L;
        const T* pex = static_cast<const T*>(o->p_exact);
        double nrm_exact = 0.0;
        if (pex) {
            TRY(Ops<T>::reduce(HRED_DOT, nullptr, N, pex, pex, 0.0, &nrm_exact, s));
            nrm_exact = std::sqrt(nrm_exact);
        }
        Count cnt;
        int nrec = 0;
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
        TRY(Ops<T>::lincomb(N, xp, 1.0, x0, 0.0, nullptr, 0.0, nullptr, nullptr, 0, s));
        TRY(fwd(fp, xp, Hxp, s));
        ++cnt.nfwd;
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
            ++cnt.nadj;
            bool recursive = false;
            if (nl > 1 && o->recursion && k > 1) {
                // grad F_rho(y) (Eq. (Twentyone)) into z; R grad F_rho into the first coarse level
                TRY(Ops<T>::lincomb(N, z, 1.0, g, 0.0, nullptr, 0.0, nullptr, nullptr, 0, s));
                TRY(Ops<T>::tv_smooth_grad(&gf, y, rho, z, lam, 1.0, s));
                TRY(Ops<T>::restrict_(&gf, z, lv[1].rg, s));
                double nRg = 0.0, ngF = 0.0;
                TRY(norm(lv[1].rg, lv[1].N, &nRg));
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
                // x = y + P (x_{h-1,*} - x_{h-1,0}), the coarse levels below solved recursively
                TRY(coarse_step(lv, nl, 1, &gf, y, nullptr, o, &cnt, s));
                TRY(Ops<T>::lincomb(N, x, 1.0, y, 0.0, nullptr, 0.0, nullptr, nullptr, 0, s));
                TRY(Ops<T>::prolong(&gf, lv[1].xs, x, 1.0, 1.0, s));
            } else {
                ++K_d;
                // x = prox_{alpha g}(y - alpha grad f(y))   (Alg. 1 lines 3-4)
                TRY(Ops<T>::lincomb(N, z, 1.0, y, -alpha, g, 0.0, nullptr, nullptr, 0, s));
                TRY(Ops<T>::tv_prox(&gf, z, x, alpha * lam, o->n_tv, 1, s));
            }
            TRY(fwd(fp, x, Hx, s));
            ++cnt.nfwd;
            double F_x = 0.0, RES = 0.0;
            TRY(F_of(x, Hx, &F_x, &RES));
            double RE = NAN;
            if (pex) {
                double sq = 0.0;
                TRY(Ops<T>::reduce(HRED_SQDIFF, nullptr, N, x, pex, 0.0, &sq, s));
                RE = std::sqrt(sq) / nrm_exact;
            }
            if (cb) cb(ctx, k, recursive ? 1 : 0, F_x, RES, RE, cnt.nfwd, cnt.nadj);
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
            rep->fwd_solves = cnt.nfwd;
            rep->adj_solves = cnt.nadj;
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
    const pat_status st = pat_plan_create(&gc, c.data(), rho.data(), a0.data(), in.alpha0_is_scalar, in.y, &sc,
                                          2.0 * in.dt, Ntc, in.prec, out);
    // a smoothing fine level has a smoothing coarse level, with its own (half) cut-off radius
    if (st == PAT_OK && fine->impl->smooth) {
        const pat_status sst = pat_plan_set_smoothing(*out, 1);
        if (sst != PAT_OK) {
            const std::string msg = pat_last_error();
            pat_plan_destroy(*out);
            *out = nullptr;
            set_error(msg);
            return sst;
        }
    }
    return st;
}

pat_status pat_mg_fista_levels(pat_plan* const* levels, int nlevels, const double* L_levels, const void* data,
                               const void* x0, const pat_fista_opts* opts, void* x_out, pat_fista_report* report,
                               pat_iter_callback cb, void* cb_ctx, void* stream) {
    set_error("");
    if (!levels || nlevels < 1 || nlevels > 8 || !L_levels || !levels[0] || !data || !x0 || !opts || !x_out) {
        set_error("NULL argument or nlevels outside 1 .. 8");
        return PAT_EINVAL;
    }
    const bool rec = opts->recursion != 0 && nlevels > 1;
    if (!(L_levels[0] > 0.0) || opts->max_iter < 0 || !(opts->tv_rho > 0.0)) {
        set_error("bad options (L, tv_rho must be > 0)");
        return PAT_EINVAL;
    }
    for (int l = 1; l < nlevels; ++l) {
        const pat_plan* up = levels[l - 1];
        const pat_plan* lo = levels[l];
        if (!lo) {
            set_error("NULL level plan");
            return PAT_EINVAL;
        }
        bool ok = lo->impl->info.precision == up->impl->info.precision && lo->impl->info.Ns == up->impl->info.Ns &&
                  lo->impl->info.Nt == (up->impl->info.Nt + 1) / 2 &&
                  lo->impl->in.grid.ndim == up->impl->in.grid.ndim;
        for (int a = 0; ok && a < up->impl->in.grid.ndim; ++a)
            ok = lo->impl->in.grid.n[a] == up->impl->in.grid.n[a] / 2;
        if (!ok) {
            set_error("level " + std::to_string(l) + " is not the coarse level of level " + std::to_string(l - 1) +
                      " (use pat_plan_create_coarse)");
            return PAT_EINVAL;
        }
        if (rec && !(L_levels[l] > 0.0)) {
            set_error("L_levels must be > 0 on every level");
            return PAT_EINVAL;
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int nl = rec ? nlevels : 1;
    if (levels[0]->impl->info.precision == PAT_F32)
        return Driver<float>::run(levels, nl, L_levels, (const float*)data, (const float*)x0, opts, (float*)x_out,
                                  report, cb, cb_ctx, s);
    return Driver<double>::run(levels, nl, L_levels, (const double*)data, (const double*)x0, opts, (double*)x_out,
                               report, cb, cb_ctx, s);
}

pat_status pat_mg_fista(pat_plan* fine, pat_plan* coarse, const void* data, const void* x0,
                        const pat_fista_opts* opts, void* x_out, pat_fista_report* report, pat_iter_callback cb,
                        void* cb_ctx, void* stream) {
    set_error("");
    if (!fine || !opts) {
        set_error("NULL argument");
        return PAT_EINVAL;
    }
    if (coarse && opts->recursion && !(opts->L_coarse > 0.0)) {
        set_error("bad options (L_coarse must be > 0)");
        return PAT_EINVAL;
    }
    pat_plan* lv[2] = {fine, coarse};
    const double Ls[2] = {opts->L, opts->L_coarse};
    return pat_mg_fista_levels(lv, coarse ? 2 : 1, Ls, data, x0, opts, x_out, report, cb, cb_ctx, stream);
}

}  // extern "C"
