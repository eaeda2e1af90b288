// pat_fft.cuh -- batched shared-memory FFT along one axis (Stockham autosort, radices 2-8).
//
// The k-space method evaluates spatial derivatives globally in the Fourier domain (Sec. I,
// Sec. II.A).  Every transform in the library is built from this device routine: a CTA holds a
// batch of complex lines in shared memory and runs log_R stages of radix-R butterflies,
// ping-ponging between two buffers.  Twiddles exp(-2 pi i m / n) are an FP64-computed table
// rounded once to the working precision; the small-DFT constants are cos / sin (2 pi m / R).
#pragma once

#include "pat_internal.cuh"

namespace pat {

// cos(2 pi m / R), sin(2 pi m / R) for m in [0, R), R in {3, 5, 7}
template <int R> __device__ __forceinline__ double root_cos(int m);
template <int R> __device__ __forceinline__ double root_sin(int m);

template <> __device__ __forceinline__ double root_cos<3>(int m) { return m == 0 ? 1.0 : -0.5; }
template <> __device__ __forceinline__ double root_sin<3>(int m) {
    return m == 0 ? 0.0 : (m == 1 ? 0.8660254037844386467637 : -0.8660254037844386467637);
}
template <> __device__ __forceinline__ double root_cos<5>(int m) {
    switch (m) {
        case 0: return 1.0;
        case 1: case 4: return 0.3090169943749474241023;
        default: return -0.8090169943749474241023;
    }
}
template <> __device__ __forceinline__ double root_sin<5>(int m) {
    switch (m) {
        case 0: return 0.0;
        case 1: return 0.9510565162951535721164;
        case 2: return 0.5877852522924731291687;
        case 3: return -0.5877852522924731291687;
        default: return -0.9510565162951535721164;
    }
}
template <> __device__ __forceinline__ double root_cos<7>(int m) {
    switch (m) {
        case 0: return 1.0;
        case 1: case 6: return 0.6234898018587335305251;
        case 2: case 5: return -0.2225209339563144042889;
        default: return -0.9009688679024191262361;
    }
}
template <> __device__ __forceinline__ double root_sin<7>(int m) {
    switch (m) {
        case 0: return 0.0;
        case 1: return 0.7818314824680298087084;
        case 2: return 0.9749279121818236070181;
        case 3: return 0.4338837391175581204758;
        case 4: return -0.4338837391175581204758;
        case 5: return -0.9749279121818236070181;
        default: return -0.7818314824680298087084;
    }
}

// R-point DFT in registers.  Forward uses exp(-2 pi i / R), inverse exp(+2 pi i / R) (unscaled).
template <typename T, bool INV> __device__ __forceinline__ void dft2(cplx<T>* v) {
    cplx<T> a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}

// multiply by -i (forward) or +i (inverse)
template <typename T, bool INV> __device__ __forceinline__ cplx<T> rot90(cplx<T> a) {
    return INV ? mkc<T>(-a.y, a.x) : mkc<T>(a.y, -a.x);
}

template <typename T, bool INV> __device__ __forceinline__ void dft4(cplx<T>& v0, cplx<T>& v1, cplx<T>& v2, cplx<T>& v3) {
    cplx<T> t0 = cadd(v0, v2), t1 = csub(v0, v2);
    cplx<T> t2 = cadd(v1, v3), t3 = rot90<T, INV>(csub(v1, v3));
    v0 = cadd(t0, t2);
    v2 = csub(t0, t2);
    v1 = cadd(t1, t3);
    v3 = csub(t1, t3);
}

template <typename T, bool INV> __device__ __forceinline__ void dft8(cplx<T>* v) {
    // even / odd split: X[k] = E[k] + W^k O[k], X[k+4] = E[k] - W^k O[k]
    cplx<T> e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    cplx<T> o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<T, INV>(e0, e1, e2, e3);
    dft4<T, INV>(o0, o1, o2, o3);
    const T h = (T)0.7071067811865475244008;
    // W^1 = (h, -+h), W^2 = -+i, W^3 = (-h, -+h)
    cplx<T> w1o1 = INV ? mkc<T>(h * (o1.x - o1.y), h * (o1.x + o1.y)) : mkc<T>(h * (o1.x + o1.y), h * (o1.y - o1.x));
    cplx<T> w2o2 = rot90<T, INV>(o2);
    cplx<T> w3o3 = INV ? mkc<T>(-h * (o3.x + o3.y), h * (o3.x - o3.y)) : mkc<T>(h * (o3.y - o3.x), -h * (o3.x + o3.y));
    v[0] = cadd(e0, o0);
    v[4] = csub(e0, o0);
    v[1] = cadd(e1, w1o1);
    v[5] = csub(e1, w1o1);
    v[2] = cadd(e2, w2o2);
    v[6] = csub(e2, w2o2);
    v[3] = cadd(e3, w3o3);
    v[7] = csub(e3, w3o3);
}

// 16 points: even / odd split into two 8-point DFTs, X[k] = E[k] + W16^k O[k], X[k+8] = E[k] -
// W16^k O[k]; W16^k = exp(-+2 pi i k / 16) from cos(pi/8), sin(pi/8) and sqrt(1/2)
template <typename T, bool INV> __device__ __forceinline__ void dft16(cplx<T>* v) {
    cplx<T> e[8], o[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        e[r] = v[2 * r];
        o[r] = v[2 * r + 1];
    }
    dft8<T, INV>(e);
    dft8<T, INV>(o);
    const T c1 = (T)0.9238795325112867561282, s1 = (T)0.3826834323650897717285, h = (T)0.7071067811865475244008;
    // forward twiddles (cos, -sin) of 2 pi k / 16, k = 0..7; the inverse takes the conjugates
    const T wc[8] = {(T)1, c1, h, s1, (T)0, -s1, -h, -c1};
    const T ws[8] = {(T)0, s1, h, c1, (T)1, c1, h, s1};
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        cplx<T> t;
        if (k == 0) t = o[0];
        else if (k == 4) t = rot90<T, INV>(o[4]);
        else {
            const T sn = INV ? ws[k] : -ws[k];
            t = mkc<T>(o[k].x * wc[k] - o[k].y * sn, o[k].x * sn + o[k].y * wc[k]);
        }
        v[k] = cadd(e[k], t);
        v[k + 8] = csub(e[k], t);
    }
}

// odd radix R = 3, 5, 7 by the symmetric pairing X_k = A_k -+ i B_k, X_{R-k} = A_k +- i B_k
template <typename T, int R, bool INV> __device__ __forceinline__ void dft_odd(cplx<T>* v) {
    constexpr int H = (R - 1) / 2;
    cplx<T> a[H], b[H];
#pragma unroll
    for (int s = 1; s <= H; ++s) {
        a[s - 1] = cadd(v[s], v[R - s]);
        b[s - 1] = csub(v[s], v[R - s]);
    }
    cplx<T> out[R];
    out[0] = v[0];
#pragma unroll
    for (int s = 0; s < H; ++s) out[0] = cadd(out[0], a[s]);
#pragma unroll
    for (int k = 1; k <= H; ++k) {
        cplx<T> A = v[0];
        cplx<T> B = mkc<T>(0, 0);
#pragma unroll
        for (int s = 1; s <= H; ++s) {
            const int m = (s * k) % R;
            const T cs = (T)root_cos<R>(m);
            const T sn = (T)root_sin<R>(m);
            A.x += a[s - 1].x * cs;
            A.y += a[s - 1].y * cs;
            B.x += b[s - 1].x * sn;
            B.y += b[s - 1].y * sn;
        }
        const cplx<T> mIB = mkc<T>(B.y, -B.x);  // -i B
        if (!INV) {
            out[k] = cadd(A, mIB);
            out[R - k] = csub(A, mIB);
        } else {
            out[k] = csub(A, mIB);
            out[R - k] = cadd(A, mIB);
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = out[r];
}

template <typename T, int R, bool INV> __device__ __forceinline__ void dft(cplx<T>* v) {
    if constexpr (R == 2) dft2<T, INV>(v);
    else if constexpr (R == 4) dft4<T, INV>(v[0], v[1], v[2], v[3]);
    else if constexpr (R == 8) dft8<T, INV>(v);
    else if constexpr (R == 16) dft16<T, INV>(v);
    else dft_odd<T, R, INV>(v);
}

// One Stockham butterfly: j in [0, n/R), k = j mod Ns with Ns = product of the radices of earlier
// stages.  src/dst point at the line start; element e of the line lives at [e * es].
template <typename T, int R, bool INV>
__device__ __forceinline__ void stockham_bfly(const cplx<T>* __restrict__ src, cplx<T>* __restrict__ dst,
                                              int j, int k, int m, int Ns, int twstep,
                                              const cplx<T>* __restrict__ tw, int es) {
    cplx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src[(j + r * m) * es];
    if (Ns > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
            const cplx<T> w = tw[r * k * twstep];
            v[r] = INV ? cmulc(v[r], w) : cmul(v[r], w);
        }
    }
    dft<T, R, INV>(v);
    const int idxD = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[(idxD + r * Ns) * es] = v[r];
}

template <typename T, bool INV>
__device__ __forceinline__ void bfly_dispatch(int R, const cplx<T>* src, cplx<T>* dst, int j, int k, int m, int Ns,
                                              int twstep, const cplx<T>* tw, int es) {
    switch (R) {
        case 8: stockham_bfly<T, 8, INV>(src, dst, j, k, m, Ns, twstep, tw, es); break;
        case 4: stockham_bfly<T, 4, INV>(src, dst, j, k, m, Ns, twstep, tw, es); break;
        case 2: stockham_bfly<T, 2, INV>(src, dst, j, k, m, Ns, twstep, tw, es); break;
        case 3: stockham_bfly<T, 3, INV>(src, dst, j, k, m, Ns, twstep, tw, es); break;
        case 5: stockham_bfly<T, 5, INV>(src, dst, j, k, m, Ns, twstep, tw, es); break;
        default: stockham_bfly<T, 7, INV>(src, dst, j, k, m, Ns, twstep, tw, es); break;
    }
}

// Transform `nlines` contiguous lines (line l at a + l n).  Consecutive threads take consecutive
// butterflies of a line.  Returns the buffer holding the result (a or b).  The caller must
// __syncthreads() before; the routine ends synchronised.
template <typename T, bool INV>
__device__ cplx<T>* fft_rows(cplx<T>* a, cplx<T>* b, const FftAxis& ax, const cplx<T>* tw, int nlines) {
    const int n = ax.n;
    int Ns = 1;
    for (int s = 0; s < ax.nst; ++s) {
        const int R = ax.rad[s];
        const int m = n / R;
        const int twstep = n / (Ns * R);
        const int total = nlines * m;
        for (int t = threadIdx.x; t < total; t += blockDim.x) {
            int line, j, k;
            if (ax.pow2) {
                const int lgm = ax.lgn - ax.lgr[s];
                line = t >> lgm;
                j = t & (m - 1);
                k = j & (Ns - 1);
            } else {
                line = t / m;
                j = t - line * m;
                k = j % Ns;
            }
            bfly_dispatch<T, INV>(R, a + line * n, b + line * n, j, k, m, Ns, twstep, tw, 1);
        }
        __syncthreads();
        cplx<T>* tmp = a;
        a = b;
        b = tmp;
        Ns *= R;
    }
    return a;
}

// Transform `nl` interleaved lines (element e of line l at a[l + e nl]).  Consecutive threads
// take consecutive lines.  lgnl = log2(nl) when nl is a power of two, else -1.
template <typename T, bool INV>
__device__ cplx<T>* fft_cols(cplx<T>* a, cplx<T>* b, const FftAxis& ax, const cplx<T>* tw, int nl, int lgnl) {
    const int n = ax.n;
    int Ns = 1;
    for (int s = 0; s < ax.nst; ++s) {
        const int R = ax.rad[s];
        const int m = n / R;
        const int twstep = n / (Ns * R);
        const int total = nl * m;
        for (int t = threadIdx.x; t < total; t += blockDim.x) {
            int line, j;
            if (lgnl >= 0) {
                line = t & (nl - 1);
                j = t >> lgnl;
            } else {
                j = t / nl;
                line = t - j * nl;
            }
            const int k = ax.pow2 ? (j & (Ns - 1)) : (j % Ns);
            bfly_dispatch<T, INV>(R, a + line, b + line, j, k, m, Ns, twstep, tw, nl);
        }
        __syncthreads();
        cplx<T>* tmp = a;
        a = b;
        b = tmp;
        Ns *= R;
    }
    return a;
}

}  // namespace pat
