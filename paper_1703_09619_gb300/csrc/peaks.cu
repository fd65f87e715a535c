// Throughput probes of the device (p2s_measure_peaks): the FP64 and FP32 fused multiply-add
// rates and the write-only HBM bandwidth.  They are the denominators of the roofline
// fractions of the FP64 kernels (FP64 pipe), the double-word kernels (FP32 pipe) and the
// write-bound contraction (a store-only stream); the copy bandwidth and the BF16 tensor
// rate come from elsewhere.
//
// FMA probes: every thread runs kChains independent FMA chains a <- a x + y (x just below
// 1, y small, so the values stay normal and bounded), 16 unrolled rounds per iteration,
// on 8 CTAs of 256 threads per SM (2048 threads per SM, enough independent FMAs in flight
// to cover the pipe latency).  The result is stored only if it equals a value it cannot
// take, which keeps every chain live without a store per FMA.
// Write probe: 16-byte streaming stores over a buffer much larger than L2, grid-stride.
// Each probe is timed with CUDA events after one warm-up launch; the best of `reps`
// launches is kept.
#include "p2s_internal.h"

namespace p2s {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;
constexpr int kRounds = 16;

__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }

template <class T>
__global__ void __launch_bounds__(kProbeThreads) k_fma_probe(T x, T y, int iters, T* sink) {
    T a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = (T)(threadIdx.x & 7) * (T)0.125 + (T)i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < kRounds; ++r)
#pragma unroll
            for (int i = 0; i < kChains; ++i) a[i] = fma_t(a[i], x, y);
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += a[i];
    if (s == (T)-12345.0) sink[blockIdx.x] = s;  // never true: the chains stay live
}

__global__ void __launch_bounds__(kProbeThreads) k_write_probe(float4* __restrict__ p, int64_t n) {
    const float4 v = make_float4(1.f, 2.f, 3.f, 4.f);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) __stcs(p + i, v);
}

// Best CUDA-event time (ms) of `reps` launches of f after one warm-up launch.
template <class F>
cudaError_t best_ms(F f, int reps, cudaStream_t s, float* out) {
    cudaEvent_t a, b;
    cudaError_t e = cudaEventCreate(&a);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&b);
    if (e != cudaSuccess) {
        cudaEventDestroy(a);
        return e;
    }
    float best = 1e30f;
    for (int r = 0; r <= reps && e == cudaSuccess; ++r) {
        cudaEventRecord(a, s);
        f();
        e = cudaGetLastError();
        cudaEventRecord(b, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (r > 0 && ms < best) best = ms;  // launch 0 warms up
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *out = best;
    return e;
}

}  // namespace

int measure_peaks(const DeviceTables& T, int64_t write_bytes, p2s_peaks* out, cudaStream_t s) {
    if (!out || write_bytes < (int64_t(1) << 20)) return fail(P2S_ERR_ARG, "p2s_measure_peaks: NULL out or buffer below 1 MiB");
    const int grid = T.sm_count * (2048 / kProbeThreads);
    const int reps = 5;
    void* sink = nullptr;
    cudaError_t e = cudaMalloc(&sink, sizeof(double) * grid);
    if (e != cudaSuccess) return fail(P2S_ERR_OOM, "p2s_measure_peaks: sink", e);
    // FP32: 20000 iterations x 128 FMAs per thread; FP64 (about 1/64 of the FP32 rate): 300
    const int it32 = 20000, it64 = 300;
    float ms32 = 0.f, ms64 = 0.f, msw = 0.f;
    e = best_ms([&] { k_fma_probe<float><<<grid, kProbeThreads, 0, s>>>(0.9999999f, 1e-7f, it32, (float*)sink); },
                reps, s, &ms32);
    if (e == cudaSuccess)
        e = best_ms([&] { k_fma_probe<double><<<grid, kProbeThreads, 0, s>>>(0.9999999, 1e-7, it64, (double*)sink); },
                    reps, s, &ms64);
    cudaFree(sink);
    if (e != cudaSuccess) return fail(P2S_ERR_CUDA, "p2s_measure_peaks: FMA probes", e);
    void* buf = nullptr;
    const int64_t n4 = write_bytes / 16;
    e = cudaMalloc(&buf, (size_t)n4 * 16);
    if (e != cudaSuccess) return fail(P2S_ERR_OOM, "p2s_measure_peaks: write buffer", e);
    e = best_ms([&] { k_write_probe<<<grid, kProbeThreads, 0, s>>>((float4*)buf, n4); }, reps, s, &msw);
    cudaFree(buf);
    if (e != cudaSuccess) return fail(P2S_ERR_CUDA, "p2s_measure_peaks: write probe", e);
    const double fma_per_thread32 = (double)it32 * kRounds * kChains, fma_per_thread64 = (double)it64 * kRounds * kChains;
    const double threads = (double)grid * kProbeThreads;
    out->fp32_fma_tflops = 2.0 * fma_per_thread32 * threads / (ms32 * 1e-3) / 1e12;
    out->fp64_fma_tflops = 2.0 * fma_per_thread64 * threads / (ms64 * 1e-3) / 1e12;
    out->hbm_write_gbs = (double)n4 * 16 / (msw * 1e-3) / 1e9;
    out->fp32_ms = ms32;
    out->fp64_ms = ms64;
    out->write_ms = msw;
    out->write_bytes = n4 * 16;
    return P2S_OK;
}

}  // namespace p2s
