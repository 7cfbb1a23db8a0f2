// Arithmetic peak of the current GPU: the fused multiply-add throughput that bounds
// the numeric factorization when it is limited by arithmetic rather than by HBM.  The
// measured HBM bandwidth and tensor-core rates come from elsewhere; the FP64 and FP32
// FMA rates are measured here, with the same kind of kernel a STREAM-style copy is for
// bandwidth: every thread runs independent FMA chains in registers, enough warps per
// SM sub-partition to keep its FMA pipe busy, and nothing is read from memory.
#include <cuda_runtime.h>

#include "ick_internal.h"

namespace ick {
namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) fma_chains(T* out, int iters, T a, T b) {
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = T(threadIdx.x + c) * T(1e-3);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains live
}

template <typename T>
cudaError_t time_probe(int grid, int iters, T* buf, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, float* ms) {
    // a < 1 and b > 0 keep every chain finite (it converges to b / (1 - a))
    fma_chains<T><<<grid, kProbeThreads, 0, s>>>(buf, iters, T(0.999), T(1e-3));  // warm-up
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    float best = 0.f;
    for (int rep = 0; rep < 3; ++rep) {
        if ((e = cudaEventRecord(e0, s)) != cudaSuccess) return e;
        fma_chains<T><<<grid, kProbeThreads, 0, s>>>(buf, iters, T(0.999), T(1e-3));
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = cudaEventRecord(e1, s)) != cudaSuccess) return e;
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) return e;
        float t = 0.f;
        if ((e = cudaEventElapsedTime(&t, e0, e1)) != cudaSuccess) return e;
        if (rep == 0 || t < best) best = t;
    }
    *ms = best;
    return cudaSuccess;
}

}  // namespace

cudaError_t measure_fma_peak(int dtype, double* gflops, cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int grid = sms * 8;  // 8 CTAs of 8 warps per SM: 16 warps per sub-partition
    // about 10 GFLOP of FP64 (some milliseconds at the GB300 FP64 rate); FP32 runs 32x longer chains
    const int iters = dtype == IC_F32 ? 8192 * 32 : 8192;
    const size_t n = size_t(grid) * kProbeThreads;
    void* buf = nullptr;
    if ((e = cudaMalloc(&buf, n * sizeof(double))) != cudaSuccess) return e;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float ms = 0.f;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        e = dtype == IC_F32 ? time_probe<float>(grid, iters, static_cast<float*>(buf), s, e0, e1, &ms)
                            : time_probe<double>(grid, iters, static_cast<double*>(buf), s, e0, e1, &ms);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(buf);
    if (e != cudaSuccess) return e;
    const double flops = 2.0 * kChains * double(iters) * double(n);
    *gflops = ms > 0.f ? flops / (double(ms) * 1e-3) / 1e9 : 0.0;
    return cudaSuccess;
}

}  // namespace ick
