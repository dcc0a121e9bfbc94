// FP64 fused-multiply-add throughput probe (roofline denominator).
#include <cuda_runtime.h>

#include "teno_probe.h"

__global__ void __launch_bounds__(256) dfma_stream(double a, double b, int iters, double *sink)
{
    double x[8];
#pragma unroll
    for (int k = 0; k < 8; k++) x[k] = (double)(threadIdx.x + k) * 1e-3;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < 8; k++) x[k] = fma(x[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; k++) s += x[k];
    sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

extern "C" int teno_probe_dfma(int blocks, int iters, double *out_sink, double *ms,
                               int64_t *dfma_total, void *stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return 2;
    dfma_stream<<<blocks, 256, 0, s>>>(0.999999, 1e-7, iters / 4, out_sink);   // warm-up
    cudaEventRecord(e0, s);
    dfma_stream<<<blocks, 256, 0, s>>>(0.999999, 1e-7, iters, out_sink);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) return 2;
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (ms) *ms = (double)t;
    if (dfma_total) *dfma_total = (int64_t)blocks * 256 * (int64_t)iters * 8;
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}
