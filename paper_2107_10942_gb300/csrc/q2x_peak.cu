// q2x_peak.cu -- ALU peak probes (declared in include/q2x.h).
//
// A measurement aid for the roofline of the element kernels, which are bound
// by the FP64 or FP32 FMA pipes: one launch of independent FMA chains on every
// SM of the device, from which the caller forms flops / (CUDA-event time).
// Each thread runs CHAINS independent chains x <- x * a + b (|a| < 1, so the
// values stay near b / (1 - a) and never overflow or become denormal); the
// chains' sum is written only if it equals a value it never takes, so the
// work is live but nothing is stored.
#include <cuda_runtime.h>

#include "q2x.h"
#include "q2x_plan.h"

namespace {

constexpr int CHAINS = 8;
constexpr int THREADS = 256;
constexpr int CTAS_PER_SM = 4;
constexpr int UNROLL = 16;

__global__ void __launch_bounds__(THREADS) peak_dfma_kernel(int64_t iters, double* sink)
{
    double x[CHAINS];
#pragma unroll
    for (int j = 0; j < CHAINS; ++j) x[j] = 1e-3 * (double)threadIdx.x + (double)j;
    const double a = 0.9999999, b = 1e-7;
#pragma unroll 1
    for (int64_t it = 0; it < iters; it += UNROLL) {
#pragma unroll
        for (int u = 0; u < UNROLL; ++u)
#pragma unroll
            for (int j = 0; j < CHAINS; ++j) x[j] = fma(x[j], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < CHAINS; ++j) s += x[j];
    if (s == -1.0) sink[0] = s;
}

__global__ void __launch_bounds__(THREADS) peak_ffma_kernel(int64_t iters, double* sink)
{
    float x[CHAINS];
#pragma unroll
    for (int j = 0; j < CHAINS; ++j) x[j] = 1e-3f * (float)threadIdx.x + (float)j;
    const float a = 0.99999f, b = 1e-5f;
#pragma unroll 1
    for (int64_t it = 0; it < iters; it += UNROLL) {
#pragma unroll
        for (int u = 0; u < UNROLL; ++u)
#pragma unroll
            for (int j = 0; j < CHAINS; ++j) x[j] = fmaf(x[j], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < CHAINS; ++j) s += x[j];
    if (s == -1.f) sink[0] = (double)s;
}

// packed FP32 pairs: one fma.rn.f32x2 performs two FMAs (4 flops)
__global__ void __launch_bounds__(THREADS) peak_ffma2_kernel(int64_t iters, double* sink)
{
    unsigned long long x[CHAINS];
#pragma unroll
    for (int j = 0; j < CHAINS; ++j) {
        const float lo = 1e-3f * (float)threadIdx.x + (float)j, hi = lo + 0.5f;
        asm("mov.b64 %0, {%1, %2};" : "=l"(x[j]) : "f"(lo), "f"(hi));
    }
    unsigned long long a, b;
    asm("mov.b64 %0, {%1, %2};" : "=l"(a) : "f"(0.99999f), "f"(0.99998f));
    asm("mov.b64 %0, {%1, %2};" : "=l"(b) : "f"(1e-5f), "f"(2e-5f));
#pragma unroll 1
    for (int64_t it = 0; it < iters; it += UNROLL) {
#pragma unroll
        for (int u = 0; u < UNROLL; ++u)
#pragma unroll
            for (int j = 0; j < CHAINS; ++j) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[j]) : "l"(a), "l"(b));
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < CHAINS; ++j) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[j]));
        s += lo + hi;
    }
    if (s == -1.f) sink[0] = (double)s;
}

}  // namespace

extern "C" q2x_status q2x_alu_peak_probe(int kind, int64_t iters, double* sink, void* cuda_stream,
                                         double* flops)
{
    if (kind < Q2X_PEAK_DFMA || kind > Q2X_PEAK_FFMA2) return q2x_fail(nullptr, Q2X_ERR_ARG, "bad probe kind %d", kind);
    if (iters <= 0 || iters > ((int64_t)1 << 40)) return q2x_fail(nullptr, Q2X_ERR_ARG, "iters out of range");
    if (!sink || !flops) return q2x_fail(nullptr, Q2X_ERR_ARG, "sink and flops must be non-NULL");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return q2x_cuda_fail(nullptr, e, "device query");
    }
    iters = (iters + UNROLL - 1) / UNROLL * UNROLL;
    const int grid = sms * CTAS_PER_SM;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const double fmas = (double)grid * THREADS * CHAINS * (double)iters;
    if (kind == Q2X_PEAK_DFMA) {
        peak_dfma_kernel<<<grid, THREADS, 0, st>>>(iters, sink);
        *flops = 2.0 * fmas;
    } else if (kind == Q2X_PEAK_FFMA) {
        peak_ffma_kernel<<<grid, THREADS, 0, st>>>(iters, sink);
        *flops = 2.0 * fmas;
    } else {
        peak_ffma2_kernel<<<grid, THREADS, 0, st>>>(iters, sink);
        *flops = 4.0 * fmas;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return q2x_cuda_fail(nullptr, e, "probe launch");
    return Q2X_OK;
}
