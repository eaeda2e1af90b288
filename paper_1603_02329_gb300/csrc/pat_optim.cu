// pat_optim.cu -- image-space kernels of the optimisation shell (Sec. IV, Sec. V):
//   isotropic TV and its proximal map by the dual fast-gradient-projection iteration
//   (Sec. IV Eq. (proxmal)), smoothed TV and its gradient (Sec. V.B Eqs. (Thirty-two),
//   (Twentyone)), the transfer operators I_h^{h-1} = 2^-d P^T and I_{h-1}^h = P (Sec. V.A), the
//   restricted bound (Sec. V.C Eq. (constraint)), FP64 reductions and FISTA vector updates.
// Conventions: image [Nz][Ny][Nx], x fastest; D = forward differences with a zero difference at
// the last index of each axis; D^T its exact transpose.
#include <cmath>
#include <cstring>
#include <vector>

#include "pat_host.h"
#include "pat_optim.h"

namespace pat {

struct ImgDims {
    int d, n[3];
    long long N;
    long long s[3];   // strides
};

static ImgDims img_dims(const pat_grid& g) {
    ImgDims D;
    D.d = g.ndim;
    D.n[0] = g.n[0];
    D.n[1] = g.n[1];
    D.n[2] = (g.ndim == 3) ? g.n[2] : 1;
    D.N = (long long)D.n[0] * D.n[1] * D.n[2];
    D.s[0] = 1;
    D.s[1] = D.n[0];
    D.s[2] = (long long)D.n[0] * D.n[1];
    return D;
}

__device__ __forceinline__ void unflat(long long i, const ImgDims& D, int* c) {
    c[0] = (int)(i % D.n[0]);
    const long long r = i / D.n[0];
    c[1] = (int)(r % D.n[1]);
    c[2] = (int)(r / D.n[1]);
}

// ------------------------------------------------------------------------------------------
// TV pieces
// ------------------------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ T dfwd(const T* x, long long i, const int* c, const ImgDims& D, int a) {
    return (c[a] < D.n[a] - 1) ? x[i + D.s[a]] - x[i] : (T)0;
}
// (D^T q)[i] = sum_a q_a[i - s_a] [c_a >= 1] - q_a[i] [c_a <= n_a - 2]
template <typename T>
__device__ __forceinline__ T dT(const T* const* q, long long i, const int* c, const ImgDims& D) {
    T v = 0;
    for (int a = 0; a < D.d; ++a) {
        if (c[a] >= 1) v += q[a][i - D.s[a]];
        if (c[a] <= D.n[a] - 2) v -= q[a][i];
    }
    return v;
}

template <typename T> struct Fields3 {
    T* f[3];
};
template <typename T> struct CFields3 {
    const T* f[3];
};

// x(j) = P_C(z - lam D^T r)(j)
template <typename T>
__device__ __forceinline__ T prox_x(const T* z, const T* const* r, long long j, const int* c, const ImgDims& D, T lam,
                                    int nonneg) {
    const T v = z[j] - lam * dT(r, j, c, D);
    return nonneg ? fmax(v, (T)0) : v;
}

// One FGP iteration (dual of the TV prox, Sec. IV): q = Pi_{|q|<=1}(r + step D x(r)),
// r_new = q + w (q - q_prev).
template <typename T>
__global__ void k_fgp_iter(ImgDims D, const T* z, CFields3<T> r, CFields3<T> qprev, Fields3<T> qnew, Fields3<T> rnew,
                           T lam, T step, T w, int nonneg) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < D.N; i += (long long)gridDim.x * blockDim.x) {
        int c[3];
        unflat(i, D, c);
        const T xi = prox_x(z, r.f, i, c, D, lam, nonneg);
        T q[3];
        T nrm2 = 0;
        for (int a = 0; a < D.d; ++a) {
            T g = 0;
            if (c[a] < D.n[a] - 1) {
                int cn[3] = {c[0], c[1], c[2]};
                cn[a] += 1;
                g = prox_x(z, r.f, i + D.s[a], cn, D, lam, nonneg) - xi;
            }
            q[a] = r.f[a][i] + step * g;
            nrm2 += q[a] * q[a];
        }
        const T sc = (T)1 / fmax((T)1, sqrt(nrm2));
        for (int a = 0; a < D.d; ++a) {
            const T qa = q[a] * sc;
            qnew.f[a][i] = qa;
            rnew.f[a][i] = qa + w * (qa - qprev.f[a][i]);
        }
    }
}

template <typename T>
__global__ void k_fgp_final(ImgDims D, const T* z, CFields3<T> q, T* x, T lam, int nonneg) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < D.N; i += (long long)gridDim.x * blockDim.x) {
        int c[3];
        unflat(i, D, c);
        x[i] = prox_x(z, q.f, i, c, D, lam, nonneg);
    }
}

// v_a(j) = D_a y(j) / sqrt(|D y(j)|^2 + rho^2)
template <typename T>
__device__ __forceinline__ T vsm(const T* y, long long j, const int* c, const ImgDims& D, int a, T rho) {
    T g[3] = {0, 0, 0};
    T s = rho * rho;
    for (int b = 0; b < D.d; ++b) {
        g[b] = dfwd(y, j, c, D, b);
        s += g[b] * g[b];
    }
    return g[a] / sqrt(s);
}

// gradient of J_rho: D^T v (Sec. V.B Eq. (Twentyone)); out = beta * out + alpha * grad
template <typename T>
__global__ void k_tv_smooth_grad(ImgDims D, const T* y, T rho, T* out, T alpha, T beta) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < D.N; i += (long long)gridDim.x * blockDim.x) {
        int c[3];
        unflat(i, D, c);
        T g = 0;
        for (int a = 0; a < D.d; ++a) {
            if (c[a] >= 1) {
                int cm[3] = {c[0], c[1], c[2]};
                cm[a] -= 1;
                g += vsm(y, i - D.s[a], cm, D, a, rho);
            }
            if (c[a] <= D.n[a] - 2) g -= vsm(y, i, c, D, a, rho);
        }
        out[i] = (beta == (T)0 ? (T)0 : beta * out[i]) + alpha * g;
    }
}

// ------------------------------------------------------------------------------------------
// FP64 reductions (two passes, fixed order: deterministic)
// ------------------------------------------------------------------------------------------
enum RedOp : int { RED_DOT = 0, RED_TV = 1, RED_TVS = 2, RED_SQDIFF = 3 };

__device__ __forceinline__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    double s = 0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)((blockDim.x + 31) >> 5); ++k) s += sh[k];
    return s;
}

template <typename T>
__global__ void k_reduce(int op, ImgDims D, long long n, const T* a, const T* b, T rho, double* partial) {
    __shared__ double sh[32];
    double acc = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (op == RED_DOT) {
            acc += (double)a[i] * (double)b[i];
        } else if (op == RED_SQDIFF) {
            const double d = (double)a[i] - (double)b[i];
            acc += d * d;
        } else {
            int c[3];
            unflat(i, D, c);
            double s = 0;
            for (int k = 0; k < D.d; ++k) {
                const double g = (double)dfwd(a, i, c, D, k);
                s += g * g;
            }
            if (op == RED_TV) acc += sqrt(s);
            else acc += sqrt(s + (double)rho * (double)rho) - (double)rho;
        }
    }
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void k_reduce_final(const double* partial, int nb, double* out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0;
        for (int k = 0; k < nb; ++k) s += partial[k];
        *out = s;
    }
}

// ------------------------------------------------------------------------------------------
// grid transfer and the restricted bound
// ------------------------------------------------------------------------------------------
// R = 2^-d P^T: coarse i gathers fine 2i-1 (1/2, i >= 1), 2i (1), 2i+1 (1/2; 1 at the last
// coarse index, where P clamps) per axis.
template <typename T>
__global__ void k_restrict(ImgDims F, ImgDims C, const T* xf, T* xc) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < C.N; i += (long long)gridDim.x * blockDim.x) {
        int c[3];
        unflat(i, C, c);
        int fi[3][3];
        T fw[3][3];
        int cnt[3];
        for (int a = 0; a < 3; ++a) {
            if (a >= C.d) {
                fi[a][0] = 0;
                fw[a][0] = 1;
                cnt[a] = 1;
                continue;
            }
            int k = 0;
            if (c[a] >= 1) {
                fi[a][k] = 2 * c[a] - 1;
                fw[a][k++] = (T)0.5;
            }
            fi[a][k] = 2 * c[a];
            fw[a][k++] = (T)1;
            fi[a][k] = 2 * c[a] + 1;
            fw[a][k++] = (c[a] == C.n[a] - 1) ? (T)1 : (T)0.5;
            cnt[a] = k;
        }
        T acc = 0;
        for (int kz = 0; kz < cnt[2]; ++kz)
            for (int ky = 0; ky < cnt[1]; ++ky)
                for (int kx = 0; kx < cnt[0]; ++kx) {
                    const long long j = fi[0][kx] + F.s[1] * fi[1][ky] + F.s[2] * fi[2][kz];
                    acc += fw[0][kx] * fw[1][ky] * fw[2][kz] * xf[j];
                }
        xc[i] = acc / (T)(1 << C.d);
    }
}

// P: fine 2i <- coarse i; fine 2i+1 <- (coarse i + coarse min(i+1, nc-1)) / 2, per axis.
// out = beta * out + alpha * P xc (beta = 0 overwrites).
template <typename T>
__global__ void k_prolong(ImgDims F, ImgDims C, const T* xc, T* xf, T alpha, T beta) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < F.N; i += (long long)gridDim.x * blockDim.x) {
        int f[3];
        unflat(i, F, f);
        int ci[3][2];
        T cw[3][2];
        int cnt[3];
        for (int a = 0; a < 3; ++a) {
            if (a >= F.d) {
                ci[a][0] = 0;
                cw[a][0] = 1;
                cnt[a] = 1;
                continue;
            }
            const int k = f[a] >> 1;
            if ((f[a] & 1) == 0) {
                ci[a][0] = k;
                cw[a][0] = 1;
                cnt[a] = 1;
            } else {
                ci[a][0] = k;
                ci[a][1] = min(k + 1, C.n[a] - 1);
                cw[a][0] = cw[a][1] = (T)0.5;
                cnt[a] = 2;
            }
        }
        T acc = 0;
        for (int kz = 0; kz < cnt[2]; ++kz)
            for (int ky = 0; ky < cnt[1]; ++ky)
                for (int kx = 0; kx < cnt[0]; ++kx)
                    acc += cw[0][kx] * cw[1][ky] * cw[2][kz] * xc[ci[0][kx] + C.s[1] * ci[1][ky] + C.s[2] * ci[2][kz]];
        xf[i] = (beta == (T)0 ? (T)0 : beta * xf[i]) + alpha * acc;
    }
}

// phi_i = (R y)_i - min over fine {2i-1, 2i, 2i+1}^d (clamped) of y  (Sec. V.C)
template <typename T>
__global__ void k_coarse_bound(ImgDims F, ImgDims C, const T* y, const T* Ry, const T* b, T* phi) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < C.N; i += (long long)gridDim.x * blockDim.x) {
        int c[3];
        unflat(i, C, c);
        T m = (T)INFINITY;
        const int oz = (C.d == 3) ? 1 : 0;
        for (int dz = -oz; dz <= oz; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int fx = min(max(2 * c[0] + dx, 0), F.n[0] - 1);
                    const int fy = min(max(2 * c[1] + dy, 0), F.n[1] - 1);
                    const int fz = (C.d == 3) ? min(max(2 * c[2] + dz, 0), F.n[2] - 1) : 0;
                    const long long f = fx + F.s[1] * fy + F.s[2] * fz;
                    m = fmin(m, b ? y[f] - b[f] : y[f]);
                }
        phi[i] = Ry[i] - m;
    }
}

// ------------------------------------------------------------------------------------------
// vector updates: out = a x + b y (+ c w); optional lower bound
// ------------------------------------------------------------------------------------------
template <typename T>
__global__ void k_lincomb(long long n, T* out, T a, const T* x, T b, const T* y, T c, const T* w, const T* lower,
                          int nonneg) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        T v = a * x[i];
        if (y) v += b * y[i];
        if (w) v += c * w[i];
        if (lower) v = fmax(v, lower[i]);
        else if (nonneg) v = fmax(v, (T)0);
        out[i] = v;
    }
}

// decimate the data record in time: out[m] = in[2 m] (rows of Ns)
template <typename T> __global__ void k_decimate_rows(const T* in, T* out, int Ntc, int Ns) {
    const long long n = (long long)Ntc * Ns;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long m = i / Ns, j = i - m * Ns;
        out[i] = in[2 * m * Ns + j];
    }
}

// ------------------------------------------------------------------------------------------
// host-side launchers (internal API, pat_optim.h)
// ------------------------------------------------------------------------------------------
static int grid_for(long long n) {
    long long b = (n + 255) / 256;
    if (b > 4 * 152) b = 4 * 152;
    return (int)(b < 1 ? 1 : b);
}

template <typename T>
pat_status Ops<T>::reduce(int op, const pat_grid* g, long long n, const T* a, const T* b, double rho, double* out,
                          cudaStream_t s) {
    ImgDims D{};
    if (g) D = img_dims(*g);
    const int nb = grid_for(n);
    double* part = nullptr;
    cudaError_t e = cudaMallocAsync(&part, (nb + 1) * sizeof(double), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync (reduction)");
    k_reduce<T><<<nb, 256, 0, s>>>(op, D, n, a, b, (T)rho, part);
    k_reduce_final<<<1, 32, 0, s>>>(part, nb, part + nb);
    e = cudaMemcpyAsync(out, part + nb, sizeof(double), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(part, s);
    if (e != cudaSuccess) return cuda_fail(e, "reduction result");
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize (reduction)");
    return PAT_OK;
}

template <typename T>
pat_status Ops<T>::tv_prox(const pat_grid* g, const T* z, T* x, double lam, int n_inner, int nonneg, cudaStream_t s) {
    const ImgDims D = img_dims(*g);
    const int nb = grid_for(D.N);
    if (!(lam > 0.0) || n_inner <= 0) {
        k_lincomb<T><<<nb, 256, 0, s>>>(D.N, x, (T)1, z, (T)0, nullptr, (T)0, nullptr, nullptr, nonneg);
        return PAT_OK;
    }
    T* buf = nullptr;
    const size_t fb = (size_t)D.N * sizeof(T);
    cudaError_t e = cudaMallocAsync(&buf, 4 * 3 * fb, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync (TV prox)");
    cudaMemsetAsync(buf, 0, 4 * 3 * fb, s);
    T* R0[3];
    T* R1[3];
    T* Q0[3];
    T* Q1[3];
    for (int a = 0; a < 3; ++a) {
        R0[a] = buf + (size_t)(0 * 3 + a) * D.N;
        R1[a] = buf + (size_t)(1 * 3 + a) * D.N;
        Q0[a] = buf + (size_t)(2 * 3 + a) * D.N;
        Q1[a] = buf + (size_t)(3 * 3 + a) * D.N;
    }
    const double step = 1.0 / (4.0 * D.d * lam);
    double t = 1.0;
    T** r = R0;
    T** rn = R1;
    T** qp = Q0;
    T** qn = Q1;
    for (int it = 0; it < n_inner; ++it) {
        const double tn = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t * t));
        const double w = (t - 1.0) / tn;
        CFields3<T> cr{{r[0], r[1], r[2]}};
        CFields3<T> cq{{qp[0], qp[1], qp[2]}};
        Fields3<T> fq{{qn[0], qn[1], qn[2]}};
        Fields3<T> fr{{rn[0], rn[1], rn[2]}};
        k_fgp_iter<T><<<nb, 256, 0, s>>>(D, z, cr, cq, fq, fr, (T)lam, (T)step, (T)w, nonneg);
        std::swap(r, rn);
        std::swap(qp, qn);
        t = tn;
    }
    CFields3<T> cq{{qp[0], qp[1], qp[2]}};
    k_fgp_final<T><<<nb, 256, 0, s>>>(D, z, cq, x, (T)lam, nonneg);
    cudaFreeAsync(buf, s);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "TV prox kernels");
    return PAT_OK;
}

template <typename T>
pat_status Ops<T>::tv_smooth_grad(const pat_grid* g, const T* y, double rho, T* out, double alpha, double beta,
                                  cudaStream_t s) {
    const ImgDims D = img_dims(*g);
    k_tv_smooth_grad<T><<<grid_for(D.N), 256, 0, s>>>(D, y, (T)rho, out, (T)alpha, (T)beta);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PAT_OK : cuda_fail(e, "smoothed TV gradient");
}

static pat_grid coarse_of(const pat_grid& f) {
    pat_grid c = f;
    for (int a = 0; a < f.ndim; ++a) c.n[a] = f.n[a] / 2;
    return c;
}

template <typename T> pat_status Ops<T>::restrict_(const pat_grid* fine, const T* xf, T* xc, cudaStream_t s) {
    const ImgDims F = img_dims(*fine), C = img_dims(coarse_of(*fine));
    k_restrict<T><<<grid_for(C.N), 256, 0, s>>>(F, C, xf, xc);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PAT_OK : cuda_fail(e, "restriction");
}

template <typename T>
pat_status Ops<T>::prolong(const pat_grid* fine, const T* xc, T* xf, double alpha, double beta, cudaStream_t s) {
    const ImgDims F = img_dims(*fine), C = img_dims(coarse_of(*fine));
    k_prolong<T><<<grid_for(F.N), 256, 0, s>>>(F, C, xc, xf, (T)alpha, (T)beta);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PAT_OK : cuda_fail(e, "prolongation");
}

template <typename T>
pat_status Ops<T>::coarse_bound(const pat_grid* fine, const T* y, T* phi, T* tmp, cudaStream_t s, const T* b) {
    const ImgDims F = img_dims(*fine), C = img_dims(coarse_of(*fine));
    k_restrict<T><<<grid_for(C.N), 256, 0, s>>>(F, C, y, tmp);
    k_coarse_bound<T><<<grid_for(C.N), 256, 0, s>>>(F, C, y, tmp, b, phi);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PAT_OK : cuda_fail(e, "coarse bound");
}

template <typename T>
pat_status Ops<T>::lincomb(long long n, T* out, double a, const T* x, double b, const T* y, double c, const T* w,
                           const T* lower, int nonneg, cudaStream_t s) {
    k_lincomb<T><<<grid_for(n), 256, 0, s>>>(n, out, (T)a, x, (T)b, y, (T)c, w, lower, nonneg);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PAT_OK : cuda_fail(e, "vector update");
}

template <typename T> pat_status Ops<T>::decimate_rows(const T* in, T* out, int Ntc, int Ns, cudaStream_t s) {
    k_decimate_rows<T><<<grid_for((long long)Ntc * Ns), 256, 0, s>>>(in, out, Ntc, Ns);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PAT_OK : cuda_fail(e, "data decimation");
}

template struct Ops<float>;
template struct Ops<double>;

static pat_status check_img_grid(const pat_grid* g) {
    if (!g || (g->ndim != 2 && g->ndim != 3)) {
        set_error("bad grid");
        return PAT_EINVAL;
    }
    for (int a = 0; a < g->ndim; ++a)
        if (g->n[a] < 1) {
            set_error("bad grid size");
            return PAT_EINVAL;
        }
    return PAT_OK;
}

static long long img_count(const pat_grid* g) {
    long long n = 1;
    for (int a = 0; a < g->ndim; ++a) n *= g->n[a];
    return n;
}

}  // namespace pat

using namespace pat;

extern "C" {

pat_status pat_tv_prox(const pat_grid* grid, const void* z, void* x, double weight, int n_inner, int nonneg,
                       pat_precision prec, void* stream) {
    set_error("");
    pat_status st = check_img_grid(grid);
    if (st != PAT_OK) return st;
    if (!z || !x || n_inner < 0) {
        set_error("bad arguments");
        return PAT_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (prec == PAT_F32) return Ops<float>::tv_prox(grid, (const float*)z, (float*)x, weight, n_inner, nonneg, s);
    return Ops<double>::tv_prox(grid, (const double*)z, (double*)x, weight, n_inner, nonneg, s);
}

pat_status pat_tv(const pat_grid* grid, const void* x, double rho, double* value, pat_precision prec, void* stream) {
    set_error("");
    pat_status st = check_img_grid(grid);
    if (st != PAT_OK) return st;
    if (!x || !value) {
        set_error("bad arguments");
        return PAT_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int op = (rho > 0.0) ? RED_TVS : RED_TV;
    if (prec == PAT_F32) return Ops<float>::reduce(op, grid, img_count(grid), (const float*)x, nullptr, rho, value, s);
    return Ops<double>::reduce(op, grid, img_count(grid), (const double*)x, nullptr, rho, value, s);
}

pat_status pat_tv_smooth_grad(const pat_grid* grid, const void* y, double rho, void* grad, pat_precision prec,
                              void* stream) {
    set_error("");
    pat_status st = check_img_grid(grid);
    if (st != PAT_OK) return st;
    if (!y || !grad || !(rho > 0.0)) {
        set_error("bad arguments");
        return PAT_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (prec == PAT_F32) return Ops<float>::tv_smooth_grad(grid, (const float*)y, rho, (float*)grad, 1.0, 0.0, s);
    return Ops<double>::tv_smooth_grad(grid, (const double*)y, rho, (double*)grad, 1.0, 0.0, s);
}

static pat_status check_even(const pat_grid* g) {
    for (int a = 0; a < g->ndim; ++a)
        if (g->n[a] < 2 || (g->n[a] & 1)) {
            set_error("fine grid sizes must be even");
            return PAT_EINVAL;
        }
    return PAT_OK;
}

pat_status pat_restrict(const pat_grid* fine, const void* xf, void* xc, pat_precision prec, void* stream) {
    set_error("");
    pat_status st = check_img_grid(fine);
    if (st == PAT_OK) st = check_even(fine);
    if (st != PAT_OK) return st;
    if (!xf || !xc) {
        set_error("NULL argument");
        return PAT_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (prec == PAT_F32) return Ops<float>::restrict_(fine, (const float*)xf, (float*)xc, s);
    return Ops<double>::restrict_(fine, (const double*)xf, (double*)xc, s);
}

pat_status pat_prolong(const pat_grid* fine, const void* xc, void* xf, pat_precision prec, void* stream) {
    set_error("");
    pat_status st = check_img_grid(fine);
    if (st == PAT_OK) st = check_even(fine);
    if (st != PAT_OK) return st;
    if (!xf || !xc) {
        set_error("NULL argument");
        return PAT_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (prec == PAT_F32) return Ops<float>::prolong(fine, (const float*)xc, (float*)xf, 1.0, 0.0, s);
    return Ops<double>::prolong(fine, (const double*)xc, (double*)xf, 1.0, 0.0, s);
}

pat_status pat_coarse_bound(const pat_grid* fine, const void* y, void* phi, pat_precision prec, void* stream) {
    set_error("");
    pat_status st = check_img_grid(fine);
    if (st == PAT_OK) st = check_even(fine);
    if (st != PAT_OK) return st;
    if (!y || !phi) {
        set_error("NULL argument");
        return PAT_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const long long nc = img_count(fine) >> fine->ndim;
    const size_t eb = (prec == PAT_F32) ? 4 : 8;
    void* tmp = nullptr;
    cudaError_t e = cudaMallocAsync(&tmp, nc * eb, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync (bound)");
    if (prec == PAT_F32) st = Ops<float>::coarse_bound(fine, (const float*)y, (float*)phi, (float*)tmp, s);
    else st = Ops<double>::coarse_bound(fine, (const double*)y, (double*)phi, (double*)tmp, s);
    cudaFreeAsync(tmp, s);
    return st;
}

pat_status pat_dot(const void* a, const void* b, int64_t n, pat_precision prec, double* out, void* stream) {
    set_error("");
    if (!a || !b || !out || n < 0) {
        set_error("bad arguments");
        return PAT_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (prec == PAT_F32) return Ops<float>::reduce(RED_DOT, nullptr, n, (const float*)a, (const float*)b, 0.0, out, s);
    return Ops<double>::reduce(RED_DOT, nullptr, n, (const double*)a, (const double*)b, 0.0, out, s);
}

}  // extern "C"
