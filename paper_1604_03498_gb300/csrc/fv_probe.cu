// Throughput probes of the SM units the plain FP32 form and the softmax use
// (instrumentation, not part of the method): scalar FP32 fused multiply-add,
// packed f32x2 fused multiply-add and the ex2.approx special function, each
// measured on every SM with long independent dependency chains and timed
// with CUDA events. They give the measured denominators of the FP32 form's
// roofline next to the one derived from unit counts and the clock.
#include <algorithm>

#include "fv_internal.h"

namespace fv {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;
constexpr int kIters = 8192;

// Target of the never-taken stores that keep the chains alive.
__device__ float g_probe_sink[kProbeThreads];

// Each thread runs kChains independent chains a <- a * b + c for kIters
// steps; the result is stored only if it is a value no chain can reach, so
// the compiler keeps every instruction.
__global__ void __launch_bounds__(kProbeThreads) probe_ffma_kernel(float b, float c, float *sink) {
    float a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = (float)(threadIdx.x + j);
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) a[j] = fmaf(a[j], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    if (s == -12345.678f) sink[threadIdx.x] = s;
}

__global__ void __launch_bounds__(kProbeThreads) probe_ffma2_kernel(float b, float c, float *sink) {
    uint64_t a[kChains], bb, cc;
    asm("mov.b64 %0, {%1, %1};" : "=l"(bb) : "f"(b));
    asm("mov.b64 %0, {%1, %1};" : "=l"(cc) : "f"(c));
#pragma unroll
    for (int j = 0; j < kChains; ++j) {
        const float v = (float)(threadIdx.x + j);
        asm("mov.b64 %0, {%1, %1};" : "=l"(a[j]) : "f"(v));
    }
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[j]) : "l"(bb), "l"(cc));
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) {
        float x, y;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(a[j]));
        s += x + y;
    }
    if (s == -12345.678f) sink[threadIdx.x] = s;
}

// a <- ex2(a) * 0.5 (converges to 1; one special-function op and one
// multiply per step)
__global__ void __launch_bounds__(kProbeThreads) probe_ex2_kernel(float *sink) {
    float a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = 0.01f * (float)(threadIdx.x & 31) + 0.1f * j;
    for (int it = 0; it < kIters / 4; ++it) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) {
            float y;
            asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a[j]));
            a[j] = y * 0.5f;
        }
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    if (s == -12345.678f) sink[threadIdx.x] = s;
}

// Best of `reps` timed launches (ms).
template <typename F>
cudaError_t best_ms(F launch, cudaStream_t st, int reps, float *best) {
    cudaEvent_t e0, e1;
    cudaError_t e;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    *best = 1e30f;
    for (int r = 0; r < reps + 1 && e == cudaSuccess; ++r) {   // the first launch warms up
        cudaEventRecord(e0, st);
        launch();
        cudaEventRecord(e1, st);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0) *best = std::min(*best, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return e;
}

}  // namespace
}  // namespace fv

using namespace fv;

extern "C" int fv_probe_peaks(double *ffma_tflops, double *ffma2_tflops, double *ex2_gops, void *cuda_stream) {
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // eight 256-thread blocks per SM: 64 warps, the most an SM holds
    const dim3 grid((unsigned)(sms * 8)), block(kProbeThreads);
    const double threads = (double)grid.x * kProbeThreads;
    float *sink = nullptr;   // never written in practice (see the kernels)
    cudaError_t e = cudaGetSymbolAddress((void **)&sink, g_probe_sink);
    if (e != cudaSuccess) return cuda_fail(e, "fv_probe_peaks: cudaGetSymbolAddress");
    float ms = 0.f;
    if (ffma_tflops) {
        e = best_ms([&] { probe_ffma_kernel<<<grid, block, 0, st>>>(0.999f, 0.001f, sink); }, st, 5, &ms);
        if (e != cudaSuccess) return cuda_fail(e, "fv_probe_peaks: FFMA probe");
        *ffma_tflops = threads * kChains * kIters * 2.0 / (ms * 1e-3) / 1e12;
    }
    if (ffma2_tflops) {
        e = best_ms([&] { probe_ffma2_kernel<<<grid, block, 0, st>>>(0.999f, 0.001f, sink); }, st, 5, &ms);
        if (e != cudaSuccess) return cuda_fail(e, "fv_probe_peaks: f32x2 FMA probe");
        *ffma2_tflops = threads * kChains * kIters * 4.0 / (ms * 1e-3) / 1e12;
    }
    if (ex2_gops) {
        e = best_ms([&] { probe_ex2_kernel<<<grid, block, 0, st>>>(sink); }, st, 5, &ms);
        if (e != cudaSuccess) return cuda_fail(e, "fv_probe_peaks: ex2 probe");
        *ex2_gops = threads * kChains * (kIters / 4) / (ms * 1e-3) / 1e9;
    }
    return FV_OK;
}
