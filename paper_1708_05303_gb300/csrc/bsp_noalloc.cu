// bsp_noalloc.cu -- triple sums over caller-provided fields without any
// device allocation.
//
// Some callers cannot call cudaMalloc: a host runtime that hands out all
// device memory from its own fixed pool (an allocation behind its back would
// break its accounting or fail once the pool holds the whole device), or an
// embedded caller with a hard memory budget that must know, when the library
// loads, every byte the library will ever hold.  bsp_triple_sums_static
// serves them: the caller passes the fields and the output, and the two
// scratch areas the reduction needs -- the triplet list and the per-segment
// partial sums -- live in file-scope device arrays of fixed size, reserved on
// every device that loads the library.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "../../include/bsp.h"
#include "bsp_internal.h"

namespace {

constexpr int NA_MAX_TRIPLETS = 1 << 17;        // 131 072 triplets (1.5 MiB of int32)
constexpr int NA_MAX_PARTIALS = 1 << 21;        // 2 097 152 FP64 partial sums (16 MiB)
constexpr int NA_MAX_DEVICES = 64;
constexpr int NA_THREADS = 256;
constexpr int NA_BLOCK = 64;                    // FP32 terms summed before the compensated fold

__device__ __align__(256) int g_na_triplets[NA_MAX_TRIPLETS * 3];
__device__ __align__(256) double g_na_partials[NA_MAX_PARTIALS];

struct NaDevice {
    bool ready = false;
    int* triplets = nullptr;
    double* partials = nullptr;
};
NaDevice g_na_dev[NA_MAX_DEVICES];
std::mutex g_na_mutex;

__device__ __forceinline__ void na_two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Block (t, seg): sum over x in segment `seg` of F_i F_j F_k for triplet t,
// FP32 products summed 64 at a time and folded into a TwoSum (hi, lo) pair
// per thread, then combined across the block in FP64 in a fixed order.
__global__ void __launch_bounds__(NA_THREADS) k_na_partial(const float* __restrict__ fields, size_t npts,
                                                         const int* __restrict__ trip, size_t seg_len,
                                                         double* __restrict__ partials) {
    __shared__ double red[NA_THREADS];
    const int t = blockIdx.x, seg = blockIdx.y;
    const float* A = fields + (size_t)trip[3 * t] * npts;
    const float* B = fields + (size_t)trip[3 * t + 1] * npts;
    const float* C = fields + (size_t)trip[3 * t + 2] * npts;
    const size_t x0 = (size_t)seg * seg_len, x1 = min(npts, x0 + seg_len);
    float acc = 0.f, hi = 0.f, lo = 0.f;
    int n = 0;
    for (size_t x = x0 + threadIdx.x; x < x1; x += NA_THREADS) {
        acc = fmaf(A[x] * B[x], C[x], acc);
        if (++n == NA_BLOCK) {
            float s, e;
            na_two_sum(hi, acc, s, e);
            hi = s;
            lo += e;
            acc = 0.f;
            n = 0;
        }
    }
    red[threadIdx.x] = (double)hi + (double)lo + (double)acc;
    __syncthreads();
    for (int o = NA_THREADS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[(size_t)t * gridDim.y + seg] = red[0];
}

__global__ void k_na_reduce(const double* __restrict__ partials, int ntrip, int nseg, double* __restrict__ T) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntrip) return;
    double s = 0.0;
    for (int k = 0; k < nseg; ++k) s += partials[(size_t)t * nseg + k];
    T[t] = s;
}

// Device addresses of the two arrays, looked up once per device with that
// device current (in host code the array names are host-side stand-ins).
bsp_status na_setup(int dev, NaDevice** out) {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    NaDevice& d = g_na_dev[dev];
    if (!d.ready) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_na_triplets);
        if (e != cudaSuccess) return bsp::record_cuda_error(e, "bsp_triple_sums_static: cudaGetSymbolAddress(triplets)");
        d.triplets = (int*)p;
        e = cudaGetSymbolAddress(&p, g_na_partials);
        if (e != cudaSuccess) return bsp::record_cuda_error(e, "bsp_triple_sums_static: cudaGetSymbolAddress(partials)");
        d.partials = (double*)p;
        d.ready = true;
    }
    *out = &d;
    return BSP_OK;
}

}  // namespace

extern "C" bsp_status bsp_triple_sums_static(const float* fields, size_t npts, int nfields,
                                             const int32_t* triplets, int ntrip, double* T, void* stream) {
    if (!fields || !T || !triplets || npts == 0 || nfields <= 0 || ntrip <= 0 ||
        (reinterpret_cast<uintptr_t>(fields) & 15u) || (reinterpret_cast<uintptr_t>(T) & 7u))
        return BSP_EINVAL;
    if (ntrip > NA_MAX_TRIPLETS) return BSP_EINVAL;
    for (int i = 0; i < 3 * ntrip; ++i)
        if (triplets[i] < 0 || triplets[i] >= nfields) return BSP_EINVAL;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return bsp::record_cuda_error(e, "bsp_triple_sums_static: cudaGetDevice");
    if (dev < 0 || dev >= NA_MAX_DEVICES) return BSP_EUNSUPPORTED;
    NaDevice* d = nullptr;
    bsp_status s = na_setup(dev, &d);
    if (s != BSP_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    e = cudaMemcpyAsync(d->triplets, triplets, sizeof(int) * 3 * (size_t)ntrip, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return bsp::record_cuda_error(e, "bsp_triple_sums_static: triplet upload");
    // segments: enough blocks to fill the GPU, each at least 4096 points,
    // and no more partial sums than the static array holds
    long long nseg = (long long)((npts + 4095) / 4096);
    nseg = std::min<long long>(nseg, 1024);
    nseg = std::min<long long>(nseg, NA_MAX_PARTIALS / ntrip);
    if (nseg < 1) nseg = 1;
    const size_t seg_len = (npts + nseg - 1) / nseg;
    // each launch reports its own error (cudaLaunchKernelEx returns it; no
    // cudaGetLastError that could pick up or clear an unrelated one)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)ntrip, (unsigned)nseg);
    cfg.blockDim = dim3(NA_THREADS);
    cfg.stream = st;
    const int* trip_dev = d->triplets;
    double* part = d->partials;
    e = cudaLaunchKernelEx(&cfg, k_na_partial, fields, npts, trip_dev, seg_len, part);
    if (e != cudaSuccess) return bsp::record_cuda_error(e, "bsp_triple_sums_static: k_na_partial launch");
    cfg.gridDim = dim3((unsigned)((ntrip + 255) / 256));
    cfg.blockDim = dim3(256);
    const double* cpart = part;
    e = cudaLaunchKernelEx(&cfg, k_na_reduce, cpart, ntrip, (int)nseg, T);
    if (e != cudaSuccess) return bsp::record_cuda_error(e, "bsp_triple_sums_static: k_na_reduce launch");
    return BSP_OK;
}
