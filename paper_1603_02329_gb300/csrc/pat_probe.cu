// pat_probe.cu -- measured FP32 FMA throughput of the device: the denominator of the instruction
// roofline of the spectral kernels (their flops are FP32 FMA and add work, no tensor-core
// contraction).  Not part of the method.
#include <algorithm>
#include <string>

#include "pat_host.h"

namespace pat {

// Eight independent FMA chains per thread (enough independent work to hide the FMA latency), `iters`
// rounds; the sum is written only when it matches an impossible value, so the work stays live.
__global__ void k_fma_probe(float a, float b, int iters, float* sink) {
    float x0 = threadIdx.x * 1e-7f, x1 = x0 + 1e-3f, x2 = x0 + 2e-3f, x3 = x0 + 3e-3f;
    float x4 = x0 + 4e-3f, x5 = x0 + 5e-3f, x6 = x0 + 6e-3f, x7 = x0 + 7e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            x0 = fmaf(x0, a, b);
            x1 = fmaf(x1, a, b);
            x2 = fmaf(x2, a, b);
            x3 = fmaf(x3, a, b);
            x4 = fmaf(x4, a, b);
            x5 = fmaf(x5, a, b);
            x6 = fmaf(x6, a, b);
            x7 = fmaf(x7, a, b);
        }
    }
    const float s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
    if (s == 1234.5678f) sink[blockIdx.x] = s;
}

}  // namespace pat

using namespace pat;

extern "C" pat_status pat_probe_fp32_peak(double* tflops, void* stream) {
    set_error("");
    if (!tflops) {
        set_error("NULL argument");
        return PAT_EINVAL;
    }
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "device attributes");
    cudaStream_t s = (cudaStream_t)stream;
    float* sink = nullptr;
    e = cudaMallocAsync(&sink, (size_t)nsm * 8 * sizeof(float), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync (probe)");
    const int blocks = nsm * 8, threads = 256, iters = 4096;
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    k_fma_probe<<<blocks, threads, 0, s>>>(0.999f, 1e-3f, 64, sink);   // warm-up
    double best = 0.0;
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
        cudaEventRecord(t0, s);
        k_fma_probe<<<blocks, threads, 0, s>>>(0.999f, 1e-3f, iters, sink);
        cudaEventRecord(t1, s);
        e = cudaEventSynchronize(t1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
        const double flops = 2.0 * 8 * 16 * (double)iters * threads * blocks;
        if (e == cudaSuccess && ms > 0.f) best = std::max(best, flops / (ms * 1e-3) / 1e12);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    cudaFreeAsync(sink, s);
    cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "FP32 probe");
    *tflops = best;
    return PAT_OK;
}
