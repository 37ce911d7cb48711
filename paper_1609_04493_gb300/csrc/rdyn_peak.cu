// rdyn_peak.cu -- FMA throughput probe (diagnostic, not on the dynamics path).
//
// Each thread runs 8 independent fused multiply-add chains so the FMA pipes,
// not the latency of one chain, set the rate. Used to report the measured
// FP32 and FP64 arithmetic peaks of the GPU next to the figures derived from
// unit counts and clocks.
#include <cuda_runtime.h>

#include "rdyn_internal.h"

namespace {

template <typename T>
__global__ void __launch_bounds__(256) fma_peak_kernel(T *out, int iters, T a, T b)
{
    T x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = T(threadIdx.x + k) * T(1e-3);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (s == T(12345.678)) out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains live
}

template <typename T>
int run(double *tflops, cudaStream_t stream)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return rd_cuda_fail(e, "rd_measure_fma_peak");
    const int blocks = sms * 8, threads = 256;
    const int iters = sizeof(T) == 4 ? 4096 : 128;
    T *out = nullptr;
    e = cudaMalloc(&out, sizeof(T) * blocks * threads);
    if (e != cudaSuccess) return rd_fail(RD_ERR_ALLOC, "rd_measure_fma_peak: %s", cudaGetErrorString(e));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(e0, stream);
        fma_peak_kernel<T><<<blocks, threads, 0, stream>>>(out, iters, T(0.999999), T(1e-7));
        cudaEventRecord(e1, stream);
        e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) break;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;  // first launch is warm-up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) return rd_cuda_fail(e, "rd_measure_fma_peak");
    const double flops = 2.0 * 8 * 16 * (double)iters * blocks * threads;
    *tflops = flops / (best * 1e-3) / 1e12;
    return RD_OK;
}

}  // namespace

extern "C" int rd_measure_fma_peak(int dtype, double *tflops, void *stream)
{
    g_rd_error.clear();
    if (!tflops) return rd_fail(RD_ERR_ARG, "rd_measure_fma_peak: null output");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (dtype == RD_F32) return run<float>(tflops, s);
    if (dtype == RD_F64) return run<double>(tflops, s);
    return rd_fail(RD_ERR_DTYPE, "rd_measure_fma_peak: dtype %d", dtype);
}
