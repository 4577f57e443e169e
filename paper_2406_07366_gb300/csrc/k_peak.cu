// Measured FMA throughput of the current GPU, the denominator of the
// roofline of the ALU-bound kernels (the short range: float32 arithmetic
// and special functions, no dense contraction).  Each thread runs eight
// independent fused multiply-add chains, so the pipe, not the latency of one
// chain, bounds the rate; a data-dependent store keeps the work live.
#include <cuda_runtime.h>

#include "bs_internal.cuh"

namespace {

constexpr int kChains = 8, kUnroll = 16;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(T* __restrict__ sink, int iters, T a, T b)
{
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
        }
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == (T)-1.2345) sink[blockIdx.x] = s;  // never true for these inputs
}

template <typename T>
int measure(int iters, double* flops)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return BS_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return BS_ERR_CUDA;
    const int blocks = sms * 8, threads = 256;
    T* sink = nullptr;
    if (cudaMalloc(&sink, sizeof(T) * blocks) != cudaSuccess) return BS_ERR_OOM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 0.0f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // the first launch is the warm-up
        e = cudaEventRecord(e0, 0);
        k_fma_peak<T><<<blocks, threads, 0, 0>>>(sink, iters, (T)0.999999, (T)1e-7);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && (best == 0.0f || ms < best)) best = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess || best <= 0.0f) return BS_ERR_CUDA;
    const double fmas = (double)blocks * threads * iters * kUnroll * kChains;
    *flops = 2.0 * fmas / (best * 1e-3);
    return BS_OK;
}

}  // namespace

extern "C" int bs_fma_peak(int precision, double* flops_per_s)
{
    if (!flops_per_s) {
        bsw::set_last_error("null output");
        return BS_ERR_ARG;
    }
    // about 0.1 s per timed launch on a GB300 in either precision
    const int rc = precision == BS_FP64 ? measure<double>(300, flops_per_s) : measure<float>(20000, flops_per_s);
    if (rc != BS_OK) bsw::set_last_error("FMA peak measurement failed");
    return rc;
}
