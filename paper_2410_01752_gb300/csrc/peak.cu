// peak.cu — measured arithmetic rates of this GPU: the denominators of the ALU-bound
// kernels' roofline (the screening pair kernel and the l0 enumeration run on the FP32 pipe,
// the FP64 re-score on the FP64 pipe).  Every thread runs 8 independent FMA chains; the
// grid fills every SM; the loop is unrolled 16 times so that its own instructions cost
// about 1% of the issue slots; timed with CUDA events, best of five launches after one.
#include "common.cuh"

#include <algorithm>

namespace sg {
namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;

__global__ void __launch_bounds__(kPeakThreads) k_peak_f32(int iters, float a, float b, float* sink) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c);
#pragma unroll 16
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 1234.5f) *sink = s;
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_f32x2(int iters, float a, float b, float* sink) {
    unsigned long long x[kChains], av, bv;
    asm("mov.b64 %0, {%1, %1};" : "=l"(av) : "f"(a));
    asm("mov.b64 %0, {%1, %1};" : "=l"(bv) : "f"(b));
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        const float u = (float)(threadIdx.x + c), v = u + 0.5f;
        asm("mov.b64 %0, {%1, %2};" : "=l"(x[c]) : "f"(u), "f"(v));
    }
#pragma unroll 16
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int c = 0; c < kChains; ++c) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[c]) : "l"(av), "l"(bv));
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        float u, v;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(u), "=f"(v) : "l"(x[c]));
        s += u + v;
    }
    if (s == 1234.5f) *sink = s;
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_f64(int iters, double a, double b, float* sink) {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (double)(threadIdx.x + c);
#pragma unroll 16
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 1234.5) *sink = (float)s;
}

}  // namespace
}  // namespace sg

// Measured FMA throughput of the current device in TFLOP/s (an FMA counts 2 flop; a paired
// FP32 FMA, 4).  kind: 0 FP32 (fma.rn.f32), 1 paired FP32 (fma.rn.f32x2), 2 FP64.  Uses the
// legacy default stream; about 0.1 s.  Errors: SISSO_ERR_ARG, SISSO_ERR_CUDA.
extern "C" sisso_status sisso_measure_alu_peak(int kind, double* tflops) {
    using namespace sg;
    if (!tflops || kind < 0 || kind > 2) return SISSO_ERR_ARG;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    float* sink = nullptr;
    if (cudaMalloc((void**)&sink, sizeof(float)) != cudaSuccess) return SISSO_ERR_CUDA;
    const int grid = sms * 8;
    // about 16 ms per FP32 launch (80 ms FP64): the burst rate of a kernel timed alone (longer
    // launches run into the power cap, which sets the rate of a kernel inside a long step)
    const int iters = kind == 2 ? 16 : 256;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 0.0;
    for (int rep = 0; rep < 6; ++rep) {
        cudaEventRecord(e0);
        if (kind == 0) k_peak_f32<<<grid, kPeakThreads>>>(iters, 0.999999f, 1e-7f, sink);
        else if (kind == 1) k_peak_f32x2<<<grid, kPeakThreads>>>(iters, 0.999999f, 1e-7f, sink);
        else k_peak_f64<<<grid, kPeakThreads>>>(iters, 0.999999999, 1e-12, sink);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double flop = (double)grid * kPeakThreads * iters * kChains * (kind == 1 ? 4.0 : 2.0);
        if (rep > 0 && ms > 0.f) best = std::max(best, flop / (ms * 1e-3) / 1e12);     // first launch warms up
    }
    const cudaError_t e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess) return SISSO_ERR_CUDA;
    *tflops = best;
    return SISSO_OK;
}
