// peak_fma.cu -- measured FP32 and FP64 fused multiply-add throughput of the
// GPU, the denominators of the ALU-side roofline fractions the benchmark
// reports (the push kernels are bound by instruction issue rather than by
// one pipe, and the Kerr-Schild push by FP64 arithmetic).
//
// Each thread runs NCH independent FMA chains x = x * a + b for `iters`
// rounds, so the pipe never waits on a dependency; the grid fills every SM
// several times over.  The result is stored only if it is a sentinel the
// chains cannot produce, so the compiler keeps the arithmetic.  Timed with
// CUDA events on the caller's stream after one untimed launch; the clocks
// are whatever the GPU runs at (nothing here changes them).
#include <cuda_runtime.h>

#include "gcb_peak.h"

namespace {

constexpr int NCH = 8;
constexpr int TPB = 256;

template <typename T>
__global__ void __launch_bounds__(TPB) k_fma(int iters, T a, T b, T *sink)
{
    T x[NCH];
#pragma unroll
    for (int c = 0; c < NCH; ++c) x[c] = T(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < NCH; ++c) x[c] = fma(x[c], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < NCH; ++c) s += x[c];
    if (s == T(-12345.0)) sink[threadIdx.x] = s;
}

// packed FP32x2 chains (Blackwell's two-lane FFMA)
__global__ void __launch_bounds__(TPB) k_fma2(int iters, float a, float b, float *sink)
{
    float2 x[NCH];
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
    for (int c = 0; c < NCH; ++c) x[c] = make_float2((float)(threadIdx.x + c), (float)c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < NCH; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < NCH; ++c) s += x[c].x + x[c].y;
    if (s == -12345.0f) sink[threadIdx.x] = s;
}

}  // namespace

extern "C" int gcb_peak_fma(int kind, int iters, void *cuda_stream, double *tflops)
{
    if (!tflops || iters < 1 || kind < GCB_PEAK_FP32 || kind > GCB_PEAK_FP64) return 1;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 2;
    const int blocks = nsm * 16;
    void *sink = nullptr;
    if (cudaMalloc(&sink, TPB * sizeof(double)) != cudaSuccess) return 2;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float ms = 0.f;
    for (int rep = 0; rep < 2; ++rep) {     // the first launch is untimed
        cudaEventRecord(e0, st);
        if (kind == GCB_PEAK_FP32)
            k_fma<float><<<blocks, TPB, 0, st>>>(iters, 0.9999999f, 1e-7f, (float *)sink);
        else if (kind == GCB_PEAK_FP32X2)
            k_fma2<<<blocks, TPB, 0, st>>>(iters, 0.9999999f, 1e-7f, (float *)sink);
        else
            k_fma<double><<<blocks, TPB, 0, st>>>(iters, 0.9999999999, 1e-12, (double *)sink);
        cudaEventRecord(e1, st);
    }
    int rc = 0;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
        cudaGetLastError() != cudaSuccess)
        rc = 2;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (rc) return rc;
    const double lanes = kind == GCB_PEAK_FP32X2 ? 2.0 : 1.0;
    const double flops = 2.0 * lanes * NCH * (double)iters * (double)blocks * TPB;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return 0;
}
