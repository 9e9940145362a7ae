// bsp_contract.cu -- CUDA-core contraction of filtered fields and the FP64
// reduction / normalisation of its partial sums.
//
// The x-integral of Eq. Standard_ell_Estim (Sec. 3.1),
//   T^l[a; b, c] = sum_x F^l_a(x) F^0_b(x) F^0_c(x),
// is organised as a matrix product over x: rows r = (l, a), columns
// p = pairs (b, c), T[r][p] = sum_x A_r(x) P_p(x) with P_p = F^0_b F^0_c formed
// once per x and shared by every (l, a).  A work item is a tile of <= 64
// pairs times <= 64 rows; a CTA owns one work item and one contiguous
// x-segment and keeps 4 x 4 outputs per thread in registers.  FP32 sums run
// over at most 64 points; each such block sum is folded into a compensated
// (TwoSum hi + lo) FP32 pair, so the segment sum is accurate to ~eps times
// the block error, and written once to the CTA's own FP64 slot.  The reduction
// sums the per-segment partials in a fixed order in FP64 (deterministic),
// then normalises: B = T / (V n^3 N_abc) or N_abc = rint(T / n^3).
#include <algorithm>

#include "bsp_internal.h"

namespace bsp {

namespace {

constexpr int CC_THREADS = 256;
constexpr int CC_ROWS = 64;
constexpr int CC_COLS = 64;
constexpr int CC_OUT = CC_ROWS * CC_COLS;

template <typename R>
struct CCCfg;
template <>
struct CCCfg<float> {
    static constexpr int XC = 32;       // x-points staged per step
    static constexpr int BLOCK = 2;     // steps summed in plain FP32 before the compensated fold
};
template <>
struct CCCfg<double> {
    static constexpr int XC = 16;
    static constexpr int BLOCK = 1;
};

template <typename R>
__device__ __forceinline__ void ld4(const R* p, R* v);
template <>
__device__ __forceinline__ void ld4<float>(const float* p, float* v) {
    float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
template <>
__device__ __forceinline__ void ld4<double>(const double* p, double* v) {
    double2 t0 = reinterpret_cast<const double2*>(p)[0];
    double2 t1 = reinterpret_cast<const double2*>(p)[1];
    v[0] = t0.x; v[1] = t0.y; v[2] = t1.x; v[3] = t1.y;
}

// Error-free sum: s + e = a + b exactly (Knuth's TwoSum, no ordering needed).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// rows: row fields (row_fields[] index them from `rows`); the pair product of
// pair (b, c) is X_b Y_c, or X_b Y_c + Y_b X_c with `sym`, X = px + s fstride.
template <typename R>
__global__ void __launch_bounds__(CC_THREADS) k_contract_cc(const R* __restrict__ rows, const R* __restrict__ px,
                                                            const R* __restrict__ py, int sym, size_t fstride,
                                                            const Work* __restrict__ works,
                                                            const int2* __restrict__ pair_fields,
                                                            const int* __restrict__ row_fields,
                                                            size_t npts, size_t seg,
                                                            double* __restrict__ partial) {
    constexpr int XC = CCCfg<R>::XC;
    constexpr int BLOCK = CCCfg<R>::BLOCK;
    constexpr bool COMP = sizeof(R) == 4;   // compensated FP32 accumulation
    constexpr int AS = CC_ROWS + 4;         // padded row strides (multiples of 16 bytes)
    constexpr int PS = CC_COLS + 4;
    __shared__ __align__(16) R As[XC][AS];
    __shared__ __align__(16) R Ps[XC][PS];
    __shared__ __align__(16) R Fz[64][XC];
    __shared__ __align__(16) R Fy[64][XC];
    const bool two = py != px;
    __shared__ int2 pf[CC_COLS];
    __shared__ int rf[CC_ROWS];

    const Work w = works[blockIdx.x];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ty = (warp & 1) * 8 + (lane >> 2);     // rows 4*ty .. 4*ty+3
    const int tx = (warp >> 1) * 4 + (lane & 3);     // cols 4*tx .. 4*tx+3
    for (int i = tid; i < CC_COLS; i += CC_THREADS) {
        int2 v = {-1, -1};
        if (i < w.npairs) {
            v = pair_fields[w.pair0 + i];
            v.x -= w.shell_lo;
            v.y -= w.shell_lo;
        }
        pf[i] = v;
    }
    for (int i = tid; i < CC_ROWS; i += CC_THREADS) rf[i] = i < w.nrows ? row_fields[w.rowbase + i] : -1;

    const size_t x_begin = (size_t)blockIdx.y * seg;
    const size_t x_end = min(npts, x_begin + seg);

    R acc[4][4], hi[4][4], lo[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = hi[i][j] = lo[i][j] = (R)0;
    int step = 0;
    __syncthreads();

    for (size_t x0 = x_begin; x0 < x_end; x0 += XC) {
        const int nx = (int)min((size_t)XC, x_end - x0);
        for (int e = tid; e < w.nshell * XC; e += CC_THREADS) {
            const int s = e / XC, x = e % XC;
            const size_t o = (size_t)(w.shell_lo + s) * fstride + x0 + x;
            Fz[s][x] = x < nx ? px[o] : (R)0;
            if (two) Fy[s][x] = x < nx ? py[o] : (R)0;
        }
        for (int e = tid; e < CC_ROWS * XC; e += CC_THREADS) {
            const int r = e / XC, x = e % XC;
            const int f = rf[r];
            As[x][r] = (f >= 0 && x < nx) ? rows[(size_t)f * fstride + x0 + x] : (R)0;
        }
        __syncthreads();
        for (int e = tid; e < CC_COLS * XC; e += CC_THREADS) {
            const int p = e % CC_COLS, x = e / CC_COLS;
            const int2 bc = pf[p];
            R v = (R)0;
            if (bc.x >= 0) {
                if (!two) v = Fz[bc.x][x] * Fz[bc.y][x];
                else if (!sym) v = Fz[bc.x][x] * Fy[bc.y][x];
                else v = Fz[bc.x][x] * Fy[bc.y][x] + Fy[bc.x][x] * Fz[bc.y][x];
            }
            Ps[x][p] = v;
        }
        __syncthreads();
#pragma unroll 4
        for (int x = 0; x < XC; ++x) {
            R a[4], p[4];
            ld4<R>(&As[x][ty * 4], a);
            ld4<R>(&Ps[x][tx * 4], p);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], p[j], acc[i][j]);
        }
        __syncthreads();
        if (COMP && ++step == BLOCK) {
            step = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float s, e;
                    two_sum((float)hi[i][j], (float)acc[i][j], s, e);
                    hi[i][j] = (R)s;
                    lo[i][j] += (R)e;
                    acc[i][j] = (R)0;
                }
        }
    }
    double* slot = partial + ((size_t)blockIdx.x * gridDim.y + blockIdx.y) * CC_OUT;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
            slot[(size_t)(ty * 4 + i) * CC_COLS + tx * 4 + j] =
                (double)acc[i][j] + (double)hi[i][j] + (double)lo[i][j];
}


// FP32 contraction with the operands staged by asynchronous copies (cp.async,
// two stages in flight): rows A_r and pair factors X_s (and Y_s) for 32
// points land in shared memory in their natural [field][x] layout while the
// previous 32 points are multiplied.  Thread (ty, tx) owns rows ty + 16 i and
// pairs 4 tx + j (i < NI, j < 4): per 4 points it reads NI float4 of A (8 distinct
// rows per warp: conflict-free with the 36-float row stride) and 4 float4 of
// the pair products P[x][p], then does 16 NI FMAs.  Block sums of 64 points are
// folded into compensated (TwoSum) pairs, as in k_contract_cc.
constexpr int C2_XS = 32;                 // points per stage
constexpr int C2_LD = C2_XS + 4;          // row stride (floats) of the staged fields
constexpr int C2_PS = CC_COLS + 4;        // row stride of the pair products

__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

struct Cc2Smem {
    float A[2][CC_ROWS][C2_LD];
    float X[2][64][C2_LD];
    float Y[2][64][C2_LD];
    float P[C2_XS][C2_PS];
    int2 pf[CC_COLS];
    int rf[CC_ROWS];
};

// Body of the FP32 contraction for a work of at most 16 NI rows: rows fill
// from 0 and thread (ty, tx) owns rows ty + 16 i, so the row blocks i >= NI
// are empty and neither staged nor multiplied (the tiles' a-ranges give
// works of 3 x (a-range) rows, most far below 64).
template <bool TWO, bool SYM, int NI>
__device__ __forceinline__ void cc32_body(Cc2Smem& S, const Work& w, const float* __restrict__ rows,
                                          const float* __restrict__ px, const float* __restrict__ py,
                                          size_t fstride, size_t npts, size_t seg, double* __restrict__ partial) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ty = (warp & 1) * 8 + (lane >> 2);     // rows ty + 16 i
    const int tx = (warp >> 1) * 4 + (lane & 3);     // pairs 4 tx + j
    const size_t x_begin = (size_t)blockIdx.y * seg;
    const size_t x_end = min(npts, x_begin + seg);
    const int nst = x_end > x_begin ? (int)((x_end - x_begin + C2_XS - 1) / C2_XS) : 0;
    const int nsh = w.nshell;
    constexpr int NR = 16 * NI;   // staged rows

    // stage s -> buffer b: 8 chunks of 4 floats per field row, zero-filled past x_end
    auto load = [&](int st, int b) {
        const size_t x0 = x_begin + (size_t)st * C2_XS;
        const int nrow_all = NR + nsh * (TWO ? 2 : 1);
        for (int e = tid; e < nrow_all * 8; e += CC_THREADS) {
            const int r = e >> 3, ch = e & 7;
            const size_t x = x0 + 4 * ch;
            const int rem = x < x_end ? (int)min((size_t)4, x_end - x) : 0;
            const float* src;
            float* dst;
            int bytes = rem * 4;
            if (r < NR) {
                const int f = S.rf[r];
                if (f < 0) bytes = 0;
                src = rows + (size_t)max(f, 0) * fstride + (bytes ? x : 0);
                dst = &S.A[b][r][4 * ch];
            } else if (r < NR + nsh) {
                const int sh = r - NR;
                src = px + (size_t)(w.shell_lo + sh) * fstride + (bytes ? x : 0);
                dst = &S.X[b][sh][4 * ch];
            } else {
                const int sh = r - NR - nsh;
                src = py + (size_t)(w.shell_lo + sh) * fstride + (bytes ? x : 0);
                dst = &S.Y[b][sh][4 * ch];
            }
            cp_async16(dst, src, bytes);
        }
    };

    float acc[NI][4], hi[NI][4], lo[NI][4];
#pragma unroll
    for (int i = 0; i < NI; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = hi[i][j] = lo[i][j] = 0.f;
    if (nst > 0) load(0, 0);
    cp_async_commit();
    for (int st = 0; st < nst; ++st) {
        const int b = st & 1;
        if (st + 1 < nst) load(st + 1, b ^ 1);
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        // pair products of this stage, P[x][p]: four consecutive points of one
        // pair per thread (16-byte reads of the staged rows; lanes take
        // consecutive pairs, so the column writes hit distinct banks)
        for (int e = tid; e < CC_COLS * (C2_XS / 4); e += CC_THREADS) {
            const int p = e % CC_COLS, x0 = 4 * (e / CC_COLS);
            const int2 bc = S.pf[p];
            float v[4] = {0.f, 0.f, 0.f, 0.f};
            if (bc.x >= 0) {
                const float4 xb = *reinterpret_cast<const float4*>(&S.X[b][bc.x][x0]);
                const float4 rc = *reinterpret_cast<const float4*>(TWO ? &S.Y[b][bc.y][x0] : &S.X[b][bc.y][x0]);
                v[0] = xb.x * rc.x; v[1] = xb.y * rc.y; v[2] = xb.z * rc.z; v[3] = xb.w * rc.w;
                if (SYM) {
                    const float4 yb = *reinterpret_cast<const float4*>(&S.Y[b][bc.x][x0]);
                    const float4 xc = *reinterpret_cast<const float4*>(&S.X[b][bc.y][x0]);
                    v[0] = fmaf(yb.x, xc.x, v[0]); v[1] = fmaf(yb.y, xc.y, v[1]);
                    v[2] = fmaf(yb.z, xc.z, v[2]); v[3] = fmaf(yb.w, xc.w, v[3]);
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) S.P[x0 + u][p] = v[u];
        }
        __syncthreads();
#pragma unroll 2
        for (int x = 0; x < C2_XS; x += 4) {
            float4 a[NI], q[4];
#pragma unroll
            for (int i = 0; i < NI; ++i) a[i] = *reinterpret_cast<const float4*>(&S.A[b][ty + 16 * i][x]);
#pragma unroll
            for (int j = 0; j < 4; ++j) q[j] = *reinterpret_cast<const float4*>(&S.P[x + j][4 * tx]);
#pragma unroll
            for (int i = 0; i < NI; ++i) {
                const float av[4] = {a[i].x, a[i].y, a[i].z, a[i].w};
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    acc[i][0] = fmaf(av[u], (&q[u].x)[0], acc[i][0]);
                    acc[i][1] = fmaf(av[u], (&q[u].x)[1], acc[i][1]);
                    acc[i][2] = fmaf(av[u], (&q[u].x)[2], acc[i][2]);
                    acc[i][3] = fmaf(av[u], (&q[u].x)[3], acc[i][3]);
                }
            }
        }
        if (st & 1) {   // every 64 points: fold the block sums into the compensated pairs
#pragma unroll
            for (int i = 0; i < NI; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float s2, e2;
                    two_sum(hi[i][j], acc[i][j], s2, e2);
                    hi[i][j] = s2;
                    lo[i][j] += e2;
                    acc[i][j] = 0.f;
                }
        }
        __syncthreads();
    }
    cp_async_wait<0>();
    double* slot = partial + ((size_t)blockIdx.x * gridDim.y + blockIdx.y) * CC_OUT;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
            slot[(size_t)(ty + 16 * i) * CC_COLS + 4 * tx + j] =
                i < NI ? (double)acc[i][j] + (double)hi[i][j] + (double)lo[i][j] : 0.0;
}

template <bool TWO, bool SYM>
__global__ void __launch_bounds__(CC_THREADS, 2) k_contract_cc32(const float* __restrict__ rows,
                                                                 const float* __restrict__ px,
                                                                 const float* __restrict__ py, size_t fstride,
                                                                 const Work* __restrict__ works,
                                                                 const int2* __restrict__ pair_fields,
                                                                 const int* __restrict__ row_fields, size_t npts,
                                                                 size_t seg, double* __restrict__ partial) {
    extern __shared__ __align__(16) unsigned char c2_raw[];
    Cc2Smem& S = *reinterpret_cast<Cc2Smem*>(c2_raw);
    const Work w = works[blockIdx.x];
    const int tid = threadIdx.x;
    for (int i = tid; i < CC_COLS; i += CC_THREADS) {
        int2 v = {-1, -1};
        if (i < w.npairs) {
            v = pair_fields[w.pair0 + i];
            v.x -= w.shell_lo;
            v.y -= w.shell_lo;
        }
        S.pf[i] = v;
    }
    for (int i = tid; i < CC_ROWS; i += CC_THREADS) S.rf[i] = i < w.nrows ? row_fields[w.rowbase + i] : -1;
    __syncthreads();
    // row blocks of 16 that hold rows of this work (uniform over the CTA)
    switch ((w.nrows + 15) >> 4) {
        case 1: cc32_body<TWO, SYM, 1>(S, w, rows, px, py, fstride, npts, seg, partial); break;
        case 2: cc32_body<TWO, SYM, 2>(S, w, rows, px, py, fstride, npts, seg, partial); break;
        case 3: cc32_body<TWO, SYM, 3>(S, w, rows, px, py, fstride, npts, seg, partial); break;
        default: cc32_body<TWO, SYM, 4>(S, w, rows, px, py, fstride, npts, seg, partial); break;
    }
}

__global__ void k_reduce(const double* __restrict__ partial, int nsplit, size_t unit, int row_stride,
                         const BinLoc* __restrict__ loc, int nout, int nbins, const double* __restrict__ counts,
                         double scale, int mode, double* __restrict__ T_out, double* __restrict__ out,
                         ShotTerms shot) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nout) return;
    const BinLoc L = loc[i];
    // nsplit > 0: slots work*nsplit .. +nsplit; else slots L.work .. L.work + L.pad
    const int nsum = nsplit > 0 ? nsplit : L.pad;
    const size_t off = (size_t)L.work * (nsplit > 0 ? nsplit : 1) * unit + (size_t)L.row * row_stride + L.col;
    double s = 0.0;
    for (int k = 0; k < nsum; ++k) s += partial[off + (size_t)k * unit];
    if (T_out) T_out[i] = s;
    if (mode == 0) {
        out[i] = rint(s * scale);
        return;
    }
    if (mode == 2) {   // raw sums, scaled
        out[i] = s * scale;
        return;
    }
    double v = s * scale;
    if (shot.n > 0) {
        // sum over the partial sets of the shot-noise contractions, each in a fixed order
        for (int t = 0; t < shot.n; ++t) {
            double u = 0.0;
            for (int k = 0; k < nsum; ++k) u += shot.partial[t][off + (size_t)k * unit];
            v -= shot.coef[t] * u;
        }
    }
    out[i] = v / counts[i % nbins];
}

// Unit fields on the orbit representatives: w_r I_a(x_r) and I_a(x_r) for
// every shell a (grid-stride over a * nrep + r).
__global__ void k_gather_reps(const double* __restrict__ fields, size_t npts, int nsh,
                              const uint32_t* __restrict__ idx, const double* __restrict__ w, size_t nrep,
                              double* __restrict__ wrows, double* __restrict__ urows) {
    const size_t total = (size_t)nsh * nrep;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t a = i / nrep, r = i - a * nrep;
        const double v = fields[a * npts + idx[r]];
        urows[i] = v;
        wrows[i] = v * w[r];
    }
}

}  // namespace

cudaError_t launch_gather_reps(const double* fields, size_t npts, int nsh, const uint32_t* idx, const double* w,
                               size_t nrep, double* wrows, double* urows, cudaStream_t st) {
    if (nsh <= 0 || nrep == 0) return cudaSuccess;
    const size_t total = (size_t)nsh * nrep;
    const unsigned blocks = (unsigned)std::min<size_t>((total + 255) / 256, 152 * 16);
    k_gather_reps<<<blocks, 256, 0, st>>>(fields, npts, nsh, idx, w, nrep, wrows, urows);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_contract_cc(const R* rows, const R* px, const R* py, int sym, size_t fstride, const Work* works,
                               int nwork, const int2* pair_fields, const int* row_fields, size_t npts, int nsplit,
                               double* partial, cudaStream_t st) {
    constexpr int XC = CCCfg<R>::XC;
    if constexpr (sizeof(R) == 4) {
        // FP32: the pipelined kernel (segments in whole stages of C2_XS points)
        size_t seg = (npts + nsplit - 1) / nsplit;
        seg = (seg + 2 * C2_XS - 1) / (2 * C2_XS) * (2 * C2_XS);
        const bool two = py != nullptr && py != px;
        const size_t smem = sizeof(Cc2Smem);
        static bool attr[3] = {false, false, false};
        auto kern = !two ? k_contract_cc32<false, false> : sym ? k_contract_cc32<true, true>
                                                                : k_contract_cc32<true, false>;
        const int ki = !two ? 0 : sym ? 2 : 1;
        if (!attr[ki]) {   // once per variant, never inside a graph capture
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            attr[ki] = true;
        }
        dim3 grid(nwork, nsplit);
        kern<<<grid, CC_THREADS, smem, st>>>(rows, px, two ? py : px, fstride, works, pair_fields, row_fields, npts,
                                             seg, partial);
        return cudaGetLastError();
    } else {
        size_t seg = (npts + nsplit - 1) / nsplit;
        seg = (seg + XC - 1) / XC * XC;
        dim3 grid(nwork, nsplit);
        k_contract_cc<R><<<grid, CC_THREADS, 0, st>>>(rows, px, py ? py : px, sym, fstride, works, pair_fields,
                                                      row_fields, npts, seg, partial);
        return cudaGetLastError();
    }
}

template cudaError_t launch_contract_cc<float>(const float*, const float*, const float*, int, size_t, const Work*,
                                               int, const int2*, const int*, size_t, int, double*, cudaStream_t);
template cudaError_t launch_contract_cc<double>(const double*, const double*, const double*, int, size_t,
                                                const Work*, int, const int2*, const int*, size_t, int, double*,
                                                cudaStream_t);

cudaError_t launch_reduce(const double* partial, int nsplit, size_t unit, int row_stride, const BinLoc* loc,
                          int nout, int nbins, const double* counts, double scale, int mode, double* T_out,
                          double* out, cudaStream_t st, const ShotTerms* shot) {
    ShotTerms none{};
    none.n = 0;
    if (nout <= 0) return cudaSuccess;
    if (unit == 0) unit = CC_OUT;
    if (row_stride == 0) row_stride = CC_COLS;
    k_reduce<<<(nout + 255) / 256, 256, 0, st>>>(partial, nsplit, unit, row_stride, loc, nout, nbins, counts, scale,
                                                 mode, T_out, out, shot ? *shot : none);
    return cudaGetLastError();
}

}  // namespace bsp
