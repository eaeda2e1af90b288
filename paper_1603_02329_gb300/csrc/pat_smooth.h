// pat_smooth.h -- arguments of the p0 smoothing S (Sec. VI.A), see pat_smooth.cu.
#pragma once

#include "pat_internal.cuh"

namespace pat {

template <typename T> struct SmoothArgs {
    int d, nx, ny, nz;          // nz = 1 for d = 2
    FftAxis ax[3];              // the plan's FFT plans per axis (x, y, z)
    const cplx<T>* tw[3];       // and their twiddles exp(-2 pi i m / n)
    double dk[3];               // 2 pi / (n dx) per axis
    double inv_kc2;             // 1 / k_c^2, k_c = min over axes of pi / dx
    double invN;                // 1 / (nx ny nz)
    cplx<T>* Z;                 // workspace: nx ny nz complex values
};

// x <- S x in place on stream s (device pointer, the plan's precision).
template <typename T> cudaError_t smooth_apply(const SmoothArgs<T>& A, T* x, cudaStream_t s);

}  // namespace pat
