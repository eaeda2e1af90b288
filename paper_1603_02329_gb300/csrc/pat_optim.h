// pat_optim.h -- internal launchers of the optimisation-shell kernels (pat_optim.cu).
#pragma once

#include "pat_internal.cuh"

namespace pat {

enum RedOpHost : int { HRED_DOT = 0, HRED_TV = 1, HRED_TVS = 2, HRED_SQDIFF = 3 };

template <typename T> struct Ops {
    // FP64-accumulated reduction (synchronises `s`): DOT sum a b, SQDIFF sum (a - b)^2,
    // TV sum |D a|, TVS sum (sqrt(|D a|^2 + rho^2) - rho)
    static pat_status reduce(int op, const pat_grid* g, long long n, const T* a, const T* b, double rho, double* out,
                             cudaStream_t s);
    static pat_status tv_prox(const pat_grid* g, const T* z, T* x, double lam, int n_inner, int nonneg,
                              cudaStream_t s);
    // out = beta out + alpha grad J_rho(y)
    static pat_status tv_smooth_grad(const pat_grid* g, const T* y, double rho, T* out, double alpha, double beta,
                                     cudaStream_t s);
    static pat_status restrict_(const pat_grid* fine, const T* xf, T* xc, cudaStream_t s);
    // xf = beta xf + alpha P xc
    static pat_status prolong(const pat_grid* fine, const T* xc, T* xf, double alpha, double beta, cudaStream_t s);
    // phi = R y - min over the fine neighbourhood of y (of y - b when a fine bound b is given)
    static pat_status coarse_bound(const pat_grid* fine, const T* y, T* phi, T* tmp, cudaStream_t s,
                                   const T* b = nullptr);
    // out = a x + b y + c w, then max(lower, .) or max(0, .) if nonneg
    static pat_status lincomb(long long n, T* out, double a, const T* x, double b, const T* y, double c, const T* w,
                              const T* lower, int nonneg, cudaStream_t s);
    static pat_status decimate_rows(const T* in, T* out, int Ntc, int Ns, cudaStream_t s);
};

}  // namespace pat
