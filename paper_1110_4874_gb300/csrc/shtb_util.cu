// FP64 throughput microbenchmarks used to state the roofline denominator of
// the FP64-bound stages: a DFMA stream (8 independent chains per thread) and
// a warp-level f64 tensor-core MMA stream (mma.sync m8n8k4, 4 independent
// accumulators per warp).  Each is warmed up once and timed with CUDA events.
#include <cuda_runtime.h>

#include <string>

#include "shtb_internal.h"

namespace {

constexpr int kIters = 4096;
constexpr int kReps = 10;

__global__ void dfma_peak_kernel(double *out, double a, double b)
{
    double x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = threadIdx.x + i;
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = fma(x[i], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += x[i];
    if (s == 12345.678) out[0] = s;   // keeps the chains live
}

__global__ void dmma_peak_kernel(double *out, double a, double b)
{
    double acc[4][2];
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[i][0] = acc[i][1] = threadIdx.x;
    const double fa = a + threadIdx.x * 1e-9, fb = b - threadIdx.x * 1e-9;
    for (int it = 0; it < kIters / 4; ++it) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            asm volatile(
                "mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                : "+d"(acc[i][0]), "+d"(acc[i][1])
                : "d"(fa), "d"(fb));
        }
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < 4; ++i) s += acc[i][0] + acc[i][1];
    if (s == 12345.678) out[0] = s;
}

}  // namespace

int measure_fp64_peak(int device, double *dfma, double *dmma)
{
    int prev = -1;
    SHTB_CUDA_TRY(cudaGetDevice(&prev));
    if (device >= 0 && device != prev) SHTB_CUDA_TRY(cudaSetDevice(device));
    int nsm = 0;
    SHTB_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device >= 0 ? device : prev));
    double *d = nullptr;
    SHTB_CUDA_TRY(cudaMalloc(&d, 64));
    cudaEvent_t e0, e1;
    SHTB_CUDA_TRY(cudaEventCreate(&e0));
    SHTB_CUDA_TRY(cudaEventCreate(&e1));
    const int blocks = nsm * 8, threads = 256;
    float ms = 0.f;

    // warm-up long enough for the clocks to settle, then time several launches
    for (int i = 0; i < 20; ++i) dfma_peak_kernel<<<blocks, threads>>>(d, 0.999999, 1e-7);
    SHTB_CUDA_TRY(cudaGetLastError());
    SHTB_CUDA_TRY(cudaEventRecord(e0));
    for (int i = 0; i < kReps; ++i) dfma_peak_kernel<<<blocks, threads>>>(d, 0.999999, 1e-7);
    SHTB_CUDA_TRY(cudaEventRecord(e1));
    SHTB_CUDA_TRY(cudaEventSynchronize(e1));
    SHTB_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    *dfma = kReps * 2.0 * 8.0 * kIters * (double)blocks * threads / (ms * 1e-3) / 1e9;

    for (int i = 0; i < 5; ++i) dmma_peak_kernel<<<blocks, threads>>>(d, 0.999999, 1e-7);
    SHTB_CUDA_TRY(cudaGetLastError());
    SHTB_CUDA_TRY(cudaEventRecord(e0));
    for (int i = 0; i < kReps; ++i) dmma_peak_kernel<<<blocks, threads>>>(d, 0.999999, 1e-7);
    SHTB_CUDA_TRY(cudaEventRecord(e1));
    SHTB_CUDA_TRY(cudaEventSynchronize(e1));
    SHTB_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    // each mma.sync m8n8k4 is 8*8*4 FMAs for the warp
    const double warps = (double)blocks * threads / 32.0;
    *dmma = kReps * 2.0 * 256.0 * 4.0 * (kIters / 4) * warps / (ms * 1e-3) / 1e9;

    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(d);
    if (device >= 0 && device != prev) cudaSetDevice(prev);
    return SHTB_OK;
}
