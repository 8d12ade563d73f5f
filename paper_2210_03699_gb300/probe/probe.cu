// Arithmetic-throughput probes (ctr_probe.h): dependent instruction chains on all SMs.  Built as a
// library of its own (libctr_probe.so) for the benchmark's roofline denominators; not part of the
// solver library or its C ABI.
#include <cuda_runtime.h>

#include "ctr_probe.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

__global__ void ffma_kernel(float* out, int64_t iters, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x * 1e-3f + c;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(x[c]) : "f"(a), "f"(b));
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 1234.5f) out[threadIdx.x] = s;
}

__global__ void ffma2_kernel(float* out, int64_t iters, float a, float b) {
    unsigned long long x[kChains];
    unsigned long long av, bv;
    asm("mov.b64 %0, {%1, %1};" : "=l"(av) : "f"(a));
    asm("mov.b64 %0, {%1, %1};" : "=l"(bv) : "f"(b));
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        float lo = threadIdx.x * 1e-3f + c, hi = lo + 0.5f;
        asm("mov.b64 %0, {%1, %2};" : "=l"(x[c]) : "f"(lo), "f"(hi));
    }
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[c]) : "l"(av), "l"(bv));
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[c]));
        s += lo + hi;
    }
    if (s == 1234.5f) out[threadIdx.x] = s;
}

__global__ void ex2_kernel(float* out, int64_t iters) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = -1e-3f * (threadIdx.x + c);
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(x[c]));
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 1234.5f) out[threadIdx.x] = s;
}

__global__ void rsqrt_kernel(float* out, int64_t iters) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1.0f + 1e-3f * (threadIdx.x + c);
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) asm volatile("rsqrt.approx.ftz.f32 %0, %0;" : "+f"(x[c]));
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 1234.5f) out[threadIdx.x] = s;
}

__global__ void dfma_kernel(double* out, int64_t iters, double a, double b) {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x * 1e-3 + c;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(x[c]) : "d"(a), "d"(b));
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 1234.5) out[threadIdx.x] = s;
}

}  // namespace

extern "C" int ctr_probe_rate(int kind, int64_t iters, double* ops_per_s, double* seconds) {
    if (!ops_per_s || iters <= 0 || kind < CTR_PROBE_FFMA || kind > CTR_PROBE_DFMA) return -1;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -4;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -4;
    const int blocks = sms * 8;
    void* out = nullptr;
    if (cudaMalloc(&out, sizeof(double) * kThreads) != cudaSuccess) return -5;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto launch = [&](int64_t it) {
        switch (kind) {
            case CTR_PROBE_FFMA: ffma_kernel<<<blocks, kThreads>>>((float*)out, it, 0.9999f, 1e-4f); break;
            case CTR_PROBE_FFMA2: ffma2_kernel<<<blocks, kThreads>>>((float*)out, it, 0.9999f, 1e-4f); break;
            case CTR_PROBE_EX2: ex2_kernel<<<blocks, kThreads>>>((float*)out, it); break;
            case CTR_PROBE_RSQRT: rsqrt_kernel<<<blocks, kThreads>>>((float*)out, it); break;
            default: dfma_kernel<<<blocks, kThreads>>>((double*)out, it, 0.9999, 1e-4); break;
        }
    };
    const double per_thread_iter = (kind == CTR_PROBE_FFMA2) ? 2.0 * kChains : (double)kChains;
    float ms = 0.f;
    bool ok = cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
    if (ok) {
        launch(iters / 10 + 1);   // warm-up
        ok = cudaGetLastError() == cudaSuccess && cudaEventRecord(e0) == cudaSuccess;
    }
    if (ok) {
        launch(iters);
        ok = cudaGetLastError() == cudaSuccess && cudaEventRecord(e1) == cudaSuccess &&
             cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (!ok || !(ms > 0.f)) return -4;
    const double ops = (double)blocks * kThreads * per_thread_iter * (double)iters;
    *ops_per_s = ops / (ms * 1e-3);
    if (seconds) *seconds = ms * 1e-3;
    return 0;
}
