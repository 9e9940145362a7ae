// bsp_batch.cu -- many mock realisations of uneven grid sizes, and the FP64
// covariance of their multipoles (the use of mock catalogues for the
// covariance, Sec. 1 and Sec. 3.1).
//
// One plan per grid size (the bins must coincide across sizes, so that the
// multipole vectors of all mocks line up); all plans share one workspace,
// since the mocks run one after another on one stream.  For every size and
// each of two device input buffers, bsp_compute is captured once into a
// CUDA graph; a run then copies a mock's delta(k) from pinned host memory
// into one input buffer on a copy stream while the graph of the previous
// mock runs on the compute stream, and appends each B to the row matrix.
// A small autotuner times the contraction grid and the FFT batch width per
// size before capture and keeps the fastest.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "../../include/bsp.h"
#include "bsp_internal.h"

namespace {

constexpr int MAX_SIZES = 8;

__global__ void k_col_mean(const double* __restrict__ X, int m, int d, double* __restrict__ mean) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= d) return;
    double s = 0.0;
    for (int i = 0; i < m; ++i) s += X[(size_t)i * d + j];
    mean[j] = s / m;
}

// C[i][j] = sum_m (X[m][i] - mean[i]) (X[m][j] - mean[j]) / (m - 1), 32 x 32
// tiles, upper triangle computed and mirrored; fixed summation order.
__global__ void __launch_bounds__(256) k_cov(const double* __restrict__ X, const double* __restrict__ mean, int m,
                                             int d, double* __restrict__ C) {
    const int bi = blockIdx.y, bj = blockIdx.x;
    if (bj < bi) return;
    __shared__ double A[16][33], Bt[16][33];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;   // 16 x 16 threads, 2 x 2 outputs each
    double acc[2][2] = {{0, 0}, {0, 0}};
    const int i0 = bi * 32, j0 = bj * 32;
    for (int k0 = 0; k0 < m; k0 += 16) {
        for (int e = threadIdx.x; e < 16 * 32; e += 256) {
            const int kk = e / 32, c = e % 32;
            const int k = k0 + kk;
            double a = 0.0, b = 0.0;
            if (k < m && i0 + c < d) a = X[(size_t)k * d + i0 + c] - mean[i0 + c];
            if (k < m && j0 + c < d) b = X[(size_t)k * d + j0 + c] - mean[j0 + c];
            A[kk][c] = a;
            Bt[kk][c] = b;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < 16; ++kk)
#pragma unroll
            for (int u = 0; u < 2; ++u)
#pragma unroll
                for (int v = 0; v < 2; ++v) acc[u][v] = fma(A[kk][ty * 2 + u], Bt[kk][tx * 2 + v], acc[u][v]);
        __syncthreads();
    }
    for (int u = 0; u < 2; ++u)
        for (int v = 0; v < 2; ++v) {
            const int i = i0 + ty * 2 + u, j = j0 + tx * 2 + v;
            if (i < d && j < d) {
                const double c = acc[u][v] / (m - 1);
                C[(size_t)i * d + j] = c;
                C[(size_t)j * d + i] = c;
            }
        }
}

}  // namespace

struct bsp_batch {
    int nsizes = 0;
    int sizes[MAX_SIZES];
    bsp_plan* plans[MAX_SIZES] = {nullptr};
    int n_ell = 0, nbins = 0;
    size_t ws_plan = 0, in_bytes[MAX_SIZES] = {0}, in_max = 0;
    bool prepared = false;
    cudaGraphExec_t exec[MAX_SIZES][2] = {{nullptr}};
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t in_ready[2] = {nullptr, nullptr}, in_free[2] = {nullptr, nullptr};
    int prec = 0;
    int tuned_ctas[MAX_SIZES] = {0}, tuned_fb[MAX_SIZES] = {0};
    int tuned_rows[MAX_SIZES] = {0}, tuned_chunk[MAX_SIZES] = {0};   // tensor-core plans
    double tuned_ms[MAX_SIZES] = {0};
    ~bsp_batch() {
        for (int s = 0; s < nsizes; ++s) {
            for (int b = 0; b < 2; ++b)
                if (exec[s][b]) cudaGraphExecDestroy(exec[s][b]);
            bsp_plan_destroy(plans[s]);
        }
        for (int b = 0; b < 2; ++b) {
            if (in_ready[b]) cudaEventDestroy(in_ready[b]);
            if (in_free[b]) cudaEventDestroy(in_free[b]);
        }
        if (copy_stream) cudaStreamDestroy(copy_stream);
    }
};

namespace {
// workspace: [plan workspace][input buffer 0][input buffer 1][B staging]
size_t r256(size_t b) { return (b + 255) / 256 * 256; }
char* in_buf(bsp_batch* bt, void* ws, int b) { return (char*)ws + r256(bt->ws_plan) + (size_t)b * r256(bt->in_max); }
double* b_stage(bsp_batch* bt, void* ws) { return (double*)((char*)ws + r256(bt->ws_plan) + 2 * r256(bt->in_max)); }
}  // namespace

extern "C" {

bsp_status bsp_batch_create(bsp_batch** out, int n_sizes, const int* sizes, double box, int n_shells,
                            const double* edges_kf, int n_ell, const int* ells, int prec, unsigned flags) {
    if (!out || n_sizes < 1 || n_sizes > MAX_SIZES || !sizes || flags != 0) return BSP_EINVAL;
    *out = nullptr;
    bsp_batch* bt = new (std::nothrow) bsp_batch();
    if (!bt) return BSP_ENOMEM;
    bt->n_ell = n_ell;
    bt->prec = prec;
    for (int s = 0; s < n_sizes; ++s) {
        bsp_status st = bsp_plan_create(&bt->plans[s], sizes[s], box, n_shells, edges_kf, n_ell, ells, prec, 0);
        if (st != BSP_OK) {
            delete bt;
            return st;
        }
        bt->nsizes = s + 1;
        bt->sizes[s] = sizes[s];
        size_t w = 0;
        bsp_workspace_size(bt->plans[s], &w);
        bt->ws_plan = std::max(bt->ws_plan, w);
        bt->in_bytes[s] = (size_t)sizes[s] * sizes[s] * (sizes[s] / 2 + 1) * 8;
        bt->in_max = std::max(bt->in_max, bt->in_bytes[s]);
    }
    *out = bt;
    return BSP_OK;
}

void bsp_batch_destroy(bsp_batch* bt) { delete bt; }

bsp_status bsp_batch_workspace_size(const bsp_batch* bt, size_t* bytes) {
    if (!bt || !bytes) return BSP_EINVAL;
    // B staging sized for the largest candidate bin list (n_ell * all a >= b >= c triplets of <= 64 shells)
    *bytes = r256(bt->ws_plan) + 2 * r256(bt->in_max) + r256((size_t)bt->n_ell * 45760 * sizeof(double));
    return BSP_OK;
}

bsp_status bsp_batch_prepare(bsp_batch* bt, void* ws, void* stream, int autotune) {
    if (!bt || !ws || ((uintptr_t)ws & 255u)) return BSP_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    // counts once per size; the bin lists must agree so that rows line up
    for (int s = 0; s < bt->nsizes; ++s) {
        bsp_status r = bsp_counts(bt->plans[s], ws, stream);
        if (r != BSP_OK) return r;
        int nb = 0;
        bsp_plan_bins(bt->plans[s], &nb, nullptr, nullptr);
        if (s == 0) {
            bt->nbins = nb;
        } else {
            std::vector<int32_t> a0((size_t)3 * bt->nbins), a1((size_t)3 * nb);
            int n0 = 0;
            bsp_plan_bins(bt->plans[0], &n0, a0.data(), nullptr);
            bsp_plan_bins(bt->plans[s], &nb, a1.data(), nullptr);
            if (nb != bt->nbins || a0 != a1) return BSP_EINVAL;   // sizes disagree on the valid bins
        }
    }
    if ((size_t)bt->n_ell * bt->nbins > (size_t)bt->n_ell * 45760) return BSP_EINVAL;
    double* Bst = b_stage(bt, ws);
    if (cudaMemsetAsync(in_buf(bt, ws, 0), 0, 2 * r256(bt->in_max), st) != cudaSuccess) return BSP_ECUDA;
    // autotune, timed on the (zero) input: the FFT batch width, and the
    // contraction grid target (CUDA-core plans) or the tensor-core tile height
    // (tensor-core plans; the accumulation chunk stays at the library's default
    // of 64 points, the shortest: the tensor core's truncating FP32
    // accumulation loses more on longer chunks, so tuning never trades accuracy)
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return BSP_ECUDA;
    const bool tc = bt->prec != BSP_FP32;
    for (int s = 0; s < bt->nsizes; ++s) {
        int best_c = 0, best_f = 0, best_r = 0, best_k = 0;
        double best = 1e30;
        const int ctas[] = {1024, 2048, 4096};
        const int rows_opt[] = {96, 64};
        const int fbs[] = {4, 16, 64};
        const int na = autotune ? (tc ? 2 : 3) : 1;
        for (int ai = 0; ai < na; ++ai)
            for (int fi = 0; fi < (autotune ? 3 : 1); ++fi) {
                const int f = autotune ? fbs[fi] : 0;
                int c = 0, rw = 0, ck = 0;
                if (autotune && tc) {
                    rw = rows_opt[ai];
                    ck = 64;
                    if (bsp_plan_tune_tc(bt->plans[s], rw, ck) != BSP_OK) continue;
                } else if (autotune) {
                    c = ctas[ai];
                }
                if (bsp_plan_tune(bt->plans[s], c, f) != BSP_OK) continue;
                bsp_status r = BSP_OK;
                for (int rep = 0; rep < 2 && r == BSP_OK; ++rep)   // warm-up, then timed
                {
                    cudaEventRecord(e0, st);
                    r = bsp_compute(bt->plans[s], in_buf(bt, ws, 0), 0.0, ws, stream, Bst);
                    cudaEventRecord(e1, st);
                }
                if (r != BSP_OK) continue;
                if (cudaEventSynchronize(e1) != cudaSuccess) return BSP_ECUDA;
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best) {
                    best = ms;
                    best_c = c;
                    best_f = f;
                    best_r = rw;
                    best_k = ck;
                }
            }
        if (tc && autotune) bsp_plan_tune_tc(bt->plans[s], best_r, best_k);
        bsp_plan_tune(bt->plans[s], best_c, best_f);
        bt->tuned_ctas[s] = best_c;
        bt->tuned_fb[s] = best_f;
        bt->tuned_rows[s] = best_r;
        bt->tuned_chunk[s] = best_k;
        bt->tuned_ms[s] = best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // one graph per (size, input buffer)
    cudaStream_t cap;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return BSP_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return BSP_ECUDA;
    for (int s = 0; s < bt->nsizes; ++s)
        for (int b = 0; b < 2; ++b) {
            cudaGraph_t g;
            if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return BSP_ECUDA;
            bsp_status r = bsp_compute(bt->plans[s], in_buf(bt, ws, b), 0.0, ws, cap, Bst);
            if (cudaStreamEndCapture(cap, &g) != cudaSuccess || r != BSP_OK) return r != BSP_OK ? r : BSP_ECUDA;
            if (bt->exec[s][b]) cudaGraphExecDestroy(bt->exec[s][b]);
            cudaError_t e = cudaGraphInstantiate(&bt->exec[s][b], g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return BSP_ECUDA;
        }
    cudaStreamDestroy(cap);
    if (!bt->copy_stream && cudaStreamCreateWithFlags(&bt->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
        return BSP_ECUDA;
    for (int b = 0; b < 2; ++b) {
        if (!bt->in_ready[b] && cudaEventCreateWithFlags(&bt->in_ready[b], cudaEventDisableTiming) != cudaSuccess)
            return BSP_ECUDA;
        if (!bt->in_free[b] && cudaEventCreateWithFlags(&bt->in_free[b], cudaEventDisableTiming) != cudaSuccess)
            return BSP_ECUDA;
    }
    bt->prepared = true;
    return BSP_OK;
}

bsp_status bsp_batch_info(const bsp_batch* bt, int* n_bins, int* tuned_ctas, int* tuned_fb, double* tuned_ms) {
    if (!bt || !n_bins) return BSP_EINVAL;
    if (!bt->prepared) return BSP_ESTATE;
    *n_bins = bt->nbins;
    for (int s = 0; s < bt->nsizes; ++s) {
        if (tuned_ctas) tuned_ctas[s] = bt->tuned_ctas[s];
        if (tuned_fb) tuned_fb[s] = bt->tuned_fb[s];
        if (tuned_ms) tuned_ms[s] = bt->tuned_ms[s];
    }
    return BSP_OK;
}

bsp_status bsp_batch_tuning(const bsp_batch* bt, int* max_rows, int* chunk_points) {
    if (!bt) return BSP_EINVAL;
    if (!bt->prepared) return BSP_ESTATE;
    for (int s = 0; s < bt->nsizes; ++s) {
        if (max_rows) max_rows[s] = bt->tuned_rows[s];
        if (chunk_points) chunk_points[s] = bt->tuned_chunk[s];
    }
    return BSP_OK;
}

bsp_status bsp_batch_bins(const bsp_batch* bt, int32_t* abc, double* counts) {
    if (!bt) return BSP_EINVAL;
    if (!bt->prepared) return BSP_ESTATE;
    int nb = 0;
    return bsp_plan_bins(bt->plans[0], &nb, abc, counts);
}

bsp_status bsp_batch_run(bsp_batch* bt, int n_mocks, const int* size_index, const void* const* delta_host,
                         void* ws, void* stream, double* rows) {
    if (!bt || n_mocks < 0 || (n_mocks && (!size_index || !delta_host || !rows)) || !ws) return BSP_EINVAL;
    if (!bt->prepared) return BSP_ESTATE;
    for (int m = 0; m < n_mocks; ++m)
        if (size_index[m] < 0 || size_index[m] >= bt->nsizes || !delta_host[m]) return BSP_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t d = (size_t)bt->n_ell * bt->nbins;
    double* Bst = b_stage(bt, ws);
    // prime: buffers start free
    for (int b = 0; b < 2; ++b)
        if (cudaEventRecord(bt->in_free[b], st) != cudaSuccess) return BSP_ECUDA;
    for (int m = 0; m < n_mocks; ++m) {
        const int b = m & 1, s = size_index[m];
        // copy stream: wait until the graph that last read buffer b is done, then load mock m
        if (cudaStreamWaitEvent(bt->copy_stream, bt->in_free[b], 0) != cudaSuccess ||
            cudaMemcpyAsync(in_buf(bt, ws, b), delta_host[m], bt->in_bytes[s], cudaMemcpyHostToDevice,
                            bt->copy_stream) != cudaSuccess ||
            cudaEventRecord(bt->in_ready[b], bt->copy_stream) != cudaSuccess)
            return BSP_ECUDA;
        if (cudaStreamWaitEvent(st, bt->in_ready[b], 0) != cudaSuccess ||
            cudaGraphLaunch(bt->exec[s][b], st) != cudaSuccess ||
            cudaEventRecord(bt->in_free[b], st) != cudaSuccess ||
            cudaMemcpyAsync(rows + (size_t)m * d, Bst, d * sizeof(double), cudaMemcpyDeviceToDevice, st) !=
                cudaSuccess)
            return BSP_ECUDA;
    }
    return BSP_OK;
}

bsp_status bsp_covariance(int m, int d, const double* rows, double* mean, double* cov, void* stream) {
    if (m < 2 || d < 1 || !rows || !mean || !cov) return BSP_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    k_col_mean<<<(d + 255) / 256, 256, 0, st>>>(rows, m, d, mean);
    dim3 grid((d + 31) / 32, (d + 31) / 32);
    k_cov<<<grid, 256, 0, st>>>(rows, mean, m, d, cov);
    return cudaGetLastError() == cudaSuccess ? BSP_OK : BSP_ECUDA;
}

}  // extern "C"
