// peak_fma.cu -- measured FP32 and FP64 fused multiply-add throughput of the
// GPU, the denominators of the ALU-side roofline fractions the benchmark
// reports (the push kernels are bound by instruction issue rather than by
// one pipe, and the Kerr-Schild push by FP64 arithmetic), and the rate of
// scattered atomic additions (the current deposition's bound).
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

// atomic additions without return (RED).  stride 1 (coalesced): the lanes
// of a warp add to 32 consecutive elements; stride 8 (scattered): to 32
// different 32-byte sectors.  Thread g adds in round i to element
// stride g + stride 1048573 i (mod n): successive rounds walk the buffer
// (1048573 a prime; n a power of two).
template <typename T>
__global__ void __launch_bounds__(TPB) k_red(int iters, T *buf, unsigned mask, unsigned stride)
{
    const unsigned g = blockIdx.x * TPB + threadIdx.x;
    for (int i = 0; i < iters; ++i) {
        const unsigned idx = (stride * g + stride * 1048573u * (unsigned)i) & mask;
        atomicAdd(buf + idx, T(1));
    }
}

}  // namespace

extern "C" int gcb_peak_red(int dtype, int pattern, int iters, void *cuda_stream, double *gops)
{
    if (!gops || iters < 1 || (dtype != 0 && dtype != 1) || (pattern != 0 && pattern != 1))
        return 1;
    const unsigned stride = pattern == 0 ? 1u : 8u;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 2;
    const int blocks = nsm * 8;
    const size_t n = (size_t)1 << 23;           // elements (32 or 64 MB: in L2)
    const size_t es = dtype == 1 ? 8 : 4;
    void *buf = nullptr;
    if (cudaMalloc(&buf, n * es) != cudaSuccess) return 2;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float ms = 0.f;
    int rc = cudaMemsetAsync(buf, 0, n * es, st) == cudaSuccess ? 0 : 2;
    for (int rep = 0; rep < 2 && !rc; ++rep) {   // the first launch is untimed
        cudaEventRecord(e0, st);
        if (dtype == 1)
            k_red<double><<<blocks, TPB, 0, st>>>(iters, (double *)buf, (unsigned)(n - 1), stride);
        else
            k_red<float><<<blocks, TPB, 0, st>>>(iters, (float *)buf, (unsigned)(n - 1), stride);
        cudaEventRecord(e1, st);
    }
    if (rc || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || cudaGetLastError() != cudaSuccess)
        rc = 2;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    if (rc) return rc;
    *gops = (double)iters * (double)blocks * TPB / (ms * 1e-3) / 1e9;
    return 0;
}

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
