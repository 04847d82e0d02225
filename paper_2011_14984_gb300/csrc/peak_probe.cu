// Throughput probe of the arithmetic pipes the pair passes run on (the paper has no
// counterpart): scalar FP32 FMA, packed FP32 FMA (two lanes per instruction), FP64 FMA and
// the MUFU reciprocal square root.  The pair passes are bound by these pipes, not by HBM or
// the tensor cores, so the roofline of a pass is its algorithmic flop rate against the rate
// measured here on the same GPU and clocks.
//
// Every thread runs CHAINS independent dependency chains of ITERS operations; the grid fills
// every SM at full occupancy, so the issue rate, not the latency, sets the time.  The results
// are written only under a condition that is never true at run time but that the compiler
// cannot prove false, which keeps the chains alive.
#include "frost.h"
#include "frost_internal.cuh"

#include <cstdio>

namespace frost {
namespace {

constexpr int kChains = 8;
constexpr int kIters = 4096;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_probe_ffma(float seed, float *sink)
{
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = seed + (float)(threadIdx.x + c);
    const float b = 0.999999f, d = 1e-7f;
    for (int it = 0; it < kIters; ++it)
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = fmaf(a[c], b, d);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == seed * -3.0f) sink[threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_probe_ffma2(float seed, float *sink)
{
    float2 a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = make_float2(seed + (float)(threadIdx.x + c), seed - (float)c);
    const float2 b = make_float2(0.999999f, 0.999998f), d = make_float2(1e-7f, 2e-7f);
    for (int it = 0; it < kIters; ++it)
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = __ffma2_rn(a[c], b, d);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c].x + a[c].y;
    if (s == seed * -3.0f) sink[threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_probe_dfma(double seed, double *sink)
{
    double a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = seed + (double)(threadIdx.x + c);
    const double b = 0.999999999, d = 1e-12;
    for (int it = 0; it < kIters / 16; ++it)
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], b, d);
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == seed * -3.0) sink[threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_probe_rsqrt(float seed, float *sink)
{
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = seed + (float)(threadIdx.x + c);
    for (int it = 0; it < kIters / 4; ++it)
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = rsqrtf(a[c]) + 1.0f;  // stays in [1, 2]
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == seed * -3.0f) sink[threadIdx.x] = s;
}

template <class K, class... A>
float time_kernel(K kernel, int blocks, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, A... args)
{
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(e0, s);
        kernel<<<blocks, kThreads, 0, s>>>(args...);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) return -1.f;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;  // the first launch warms up
    }
    return best;
}

}  // namespace
}  // namespace frost

using namespace frost;

extern "C" frost_status frost_peak_probe(double *out, void *cuda_stream)
{
    clear_last_error();
    if (!out) {
        set_last_error("frost_peak_probe: out is NULL");
        return FROST_EINVAL;
    }
    const cudaStream_t s = (cudaStream_t)cuda_stream;
    int dev = 0, nsm = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_probe_ffma, kThreads, 0);
    if (e != cudaSuccess || nsm <= 0 || per_sm <= 0) {
        set_last_error("frost_peak_probe: device query failed: %s", cudaGetErrorString(e));
        return FROST_ECUDA;
    }
    // full occupancy, several waves so that the tail is small
    const int blocks = nsm * per_sm * 4;
    const double threads = (double)blocks * kThreads;
    void *sink = nullptr;
    e = cudaMalloc(&sink, sizeof(double) * kThreads);
    if (e != cudaSuccess) {
        set_last_error("frost_peak_probe: cudaMalloc: %s", cudaGetErrorString(e));
        return FROST_ENOMEM;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const float t_ffma = time_kernel(k_probe_ffma, blocks, s, e0, e1, 1.5f, (float *)sink);
    const float t_ffma2 = time_kernel(k_probe_ffma2, blocks, s, e0, e1, 1.5f, (float *)sink);
    const float t_dfma = time_kernel(k_probe_dfma, blocks, s, e0, e1, 1.5, (double *)sink);
    const float t_rsq = time_kernel(k_probe_rsqrt, blocks, s, e0, e1, 1.5f, (float *)sink);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    e = cudaGetLastError();
    if (e != cudaSuccess || t_ffma <= 0.f || t_ffma2 <= 0.f || t_dfma <= 0.f || t_rsq <= 0.f) {
        set_last_error("frost_peak_probe: a probe kernel failed: %s", cudaGetErrorString(e));
        return FROST_ECUDA;
    }
    const double ops = threads * kChains;
    out[0] = 2.0 * ops * kIters / (t_ffma * 1e-3) / 1e12;             // FFMA TFLOP/s
    out[1] = 4.0 * ops * kIters / (t_ffma2 * 1e-3) / 1e12;            // packed FFMA2 TFLOP/s
    out[2] = 2.0 * ops * (kIters / 16) / (t_dfma * 1e-3) / 1e12;      // DFMA TFLOP/s
    out[3] = ops * (kIters / 4) / (t_rsq * 1e-3);                     // MUFU rsqrt per second
    out[4] = (double)nsm;
    out[5] = (double)per_sm * kThreads;  // resident threads per SM in the probe
    return FROST_OK;
}
