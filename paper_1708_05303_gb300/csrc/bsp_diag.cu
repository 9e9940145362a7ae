// bsp_diag.cu -- measured FP32 CUDA-core throughput of this GPU, the peak the
// FP32 contraction's roofline is taken against.
//
// Every thread runs 8 independent FMA chains (enough instruction-level
// parallelism to hide the FMA latency with 32 warps per SM), one block of
// 1024 threads per SM, for a fixed number of iterations; the elapsed time of
// the launch (CUDA events on the caller's stream) gives the rate.  The chains
// stay bounded (x <- x * b + c with 0 < b < 1) and their sum is stored, so
// nothing is optimised away.
#include <cuda_runtime.h>

#include "bsp_internal.h"

namespace {

constexpr int DG_THREADS = 1024;
constexpr int DG_CHAINS = 8;

__global__ void __launch_bounds__(DG_THREADS) k_fma_chains(int iters, float b, float c, float* __restrict__ out) {
    float x[DG_CHAINS];
#pragma unroll
    for (int j = 0; j < DG_CHAINS; ++j) x[j] = (float)(threadIdx.x + j) * 1e-3f;
    for (int i = 0; i < iters; i += 16) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int j = 0; j < DG_CHAINS; ++j) x[j] = fmaf(x[j], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < DG_CHAINS; ++j) s += x[j];
    out[(size_t)blockIdx.x * DG_THREADS + threadIdx.x] = s;
}

}  // namespace

extern "C" bsp_status bsp_fp32_fma_peak(int iters, void* stream, float* scratch, double* tflops, double* ms) {
    if (!tflops || !scratch || iters < 16 || iters % 16 || (reinterpret_cast<uintptr_t>(scratch) & 3u))
        return BSP_EINVAL;
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return bsp::record_cuda_error(e, "bsp_fp32_fma_peak: device query");
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return bsp::record_cuda_error(e, "bsp_fp32_fma_peak: events");
    }
    // one short warm-up launch, then the timed one
    k_fma_chains<<<nsm, DG_THREADS, 0, st>>>(16 * 64, 0.999f, 1e-4f, scratch);
    cudaEventRecord(e0, st);
    k_fma_chains<<<nsm, DG_THREADS, 0, st>>>(iters, 0.999f, 1e-4f, scratch);
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return bsp::record_cuda_error(e, "bsp_fp32_fma_peak: timed launch");
    const double flop = 2.0 * DG_CHAINS * (double)iters * (double)nsm * DG_THREADS;
    *tflops = flop / (t * 1e-3) / 1e12;
    if (ms) *ms = t;
    return BSP_OK;
}
