// bsp_power.cu -- power-spectrum multipoles P^(l)(k) on the shells of a plan.
//
// Eq. PowSpecMultipole (Sec. 2): with the line of sight along z (plane-
// parallel), delta^(l)(k) delta^(0)(-k) = w_l(mu) |delta(k)|^2, and the
// average over the directions of shell a is the mean over its modes:
//   P^l_a = 1/(V N_a) sum_{n in a} w_l(mu_n) |delta(n)|^2,   w_l = (2l+1) L_l.
// The half spectrum holds each mode pair once for 0 < n_z < n/2 (weight 2)
// and both members on the n_z = 0 and n/2 planes (weight 1 each, with the
// Hermitian part (delta(n) + conj delta(-n))/2, as the real inverse FFT sees
// it).  Only |f| <= K per axis can lie in a shell, so only that box is read.
// One pass: the products w_l |delta|^2 are formed in FP32 (the input is
// FP32; GB300's FP64 rate is a small fraction of its FP32 rate), summed in
// FP64 per warp and shell, per CTA, then over CTAs in a fixed order by a
// second kernel (deterministic), which normalises.  A batch of spectra (the
// sub-cubes of the integrated bispectrum, Sec. 3.4) runs as gridDim.y, each
// spectrum's products optionally weighted by its own Re delta(0).
#include "bsp_internal.h"

namespace bsp {

namespace {

// w_l = (2l+1) L_l(mu), mu^2 = fz2/n2, from the exact integer numerators
// 3 fz2 - n2 and 35 fz2^2 - 30 fz2 n2 + 3 n2^2: a few ulp of w_l itself (not
// of 2l+1), and exactly 0 where L_l vanishes on the lattice (mu^2 = 1/3).
__device__ __forceinline__ float legendre_w(int ell, int fz2, int n2) {
    if (ell == 0) return 1.f;
    if (ell == 2) return 2.5f * (float)(3 * fz2 - n2) / (float)n2;             // 5 L_2
    const long long f = fz2, q = n2;
    const float d = (float)n2;
    return 1.125f * (float)(35 * f * f - 30 * f * q + 3 * q * q) / (d * d);    // 9 L_4
}

constexpr int PW_WARPS = 8;   // warps per CTA

// SHOT: also sum w_l per shell (the weights of the shot-noise term); without
// it those sums stay 0 and the scan carries 4 values instead of 7.
template <bool SHOT>
__global__ void __launch_bounds__(32 * PW_WARPS) k_power_partial(const cx<float>* __restrict__ delta,
                                                                 const cx<float>* __restrict__ Q, FftGeom g,
                                                                 const int16_t* __restrict__ shell_of, int nsh,
                                                                 PowerEll ells, double* __restrict__ partial,
                                                                 size_t bstride, int dc_weight, int n2top) {
    // per warp [2 nell + 1][nsh] FP64: sum w|d|^2 per l, sum w per l, mode count
    extern __shared__ double acc[];
    const int nell = ells.n, per = (2 * nell + 1) * nsh;
    for (int i = threadIdx.x; i < PW_WARPS * per; i += blockDim.x) acc[i] = 0.0;
    __syncthreads();
    const int N = g.n, H = N / 2 + 1;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double* mine = acc + (size_t)wid * per;
    // spectrum blockIdx.y of a batch; with dc_weight its products carry the
    // factor Re delta(0) of that spectrum (the cube mean of Sec. 3.4)
    delta += (size_t)blockIdx.y * bstride;
    const float dcw = dc_weight ? delta[0].re : 1.f;
    const long long rows = (long long)g.nK * g.nK;
    // one warp per row, 32 consecutive n_z at a time: along a row |n| grows with
    // n_z, so the lanes of one shell are a contiguous run; a segmented sum over
    // the run (FP32, at most 32 terms) leaves its total in the run's last lane,
    // the only writer of that shell in this warp (FP64): no atomics, and every
    // sum is taken in a fixed order
    for (long long r = (long long)blockIdx.x * PW_WARPS + wid; r < rows; r += (long long)gridDim.x * PW_WARPS) {
        const int cx_ = (int)(r / g.nK), cy = (int)(r % g.nK);
        const int fx = g.pruned ? cx_ - g.K : (cx_ < N / 2 ? cx_ : cx_ - N);
        const int fy = g.pruned ? cy - g.K : (cy < N / 2 ? cy : cy - N);
        if (fx * fx + fy * fy > n2top) continue;   // no mode of this row lies in a shell
        const int ix = (fx + N) % N, iy = (fy + N) % N;
        const cx<float>* row = delta + ((size_t)ix * N + iy) * H;
        const size_t mo = ((size_t)((N - ix) % N) * N + (N - iy) % N) * H, ro = ((size_t)ix * N + iy) * H;
        const cx<float>* mrow = delta + mo;
        for (int k0 = 0; k0 < g.nKz; k0 += 32) {
            const int kz = k0 + lane;
            int s = -1;
            float v[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (kz < g.nKz) {
                const int fz = kz == N / 2 ? -(N / 2) : kz;
                const int n2 = fx * fx + fy * fy + fz * fz;
                if (n2 > 0 && n2 <= g.n2max) s = shell_of[n2];
                if (s >= 0) {
                    const cx<float> d = row[kz];
                    float re = d.re, im = d.im, h = 2.f;
                    if (kz == 0 || kz == N / 2) {
                        const cx<float> m = mrow[kz];
                        re = 0.5f * (re + m.re);
                        im = 0.5f * (im - m.im);
                        h = 1.f;
                    }
                    float p = re * re + im * im;
                    if (Q) {   // cross spectrum: Re[conj(Q) delta], Hermitian parts on both
                        const cx<float> q = Q[ro + kz];
                        float qr = q.re, qi = q.im;
                        if (kz == 0 || kz == N / 2) {
                            const cx<float> qm = Q[mo + kz];
                            qr = 0.5f * (qr + qm.re);
                            qi = 0.5f * (qi - qm.im);
                        }
                        p = qr * re + qi * im;
                    }
                    p *= h * dcw;
                    for (int l = 0; l < nell; ++l) {
                        const float w = legendre_w(ells.ell[l], fz * fz, n2);
                        v[l] = w * p;
                        if (SHOT) v[4 + l] = w * h;
                    }
                    v[3] = h;
                }
            }
            if (__all_sync(0xffffffffu, s < 0)) continue;
            // v: [0, 3) w_l p, [3] the mode count, [4, 7) w_l (SHOT only)
            constexpr int NV = SHOT ? 7 : 4;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int so = __shfl_up_sync(0xffffffffu, s, o);
                const bool take = lane >= o && so == s;
#pragma unroll
                for (int t = 0; t < NV; ++t) {
                    const float x = __shfl_up_sync(0xffffffffu, v[t], o);
                    if (take) v[t] += x;
                }
            }
            const int snext = __shfl_down_sync(0xffffffffu, s, 1);
            if (s >= 0 && (lane == 31 || snext != s)) {
                for (int l = 0; l < nell; ++l) {
                    mine[l * nsh + s] += (double)v[l];
                    if (SHOT) mine[(nell + l) * nsh + s] += (double)v[4 + l];
                }
                mine[2 * nell * nsh + s] += (double)v[3];
            }
            __syncwarp();
        }
    }
    __syncthreads();
    double* dst = partial + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * per;
    for (int i = threadIdx.x; i < per; i += blockDim.x) {
        double t = 0.0;
        for (int w = 0; w < PW_WARPS; ++w) t += acc[(size_t)w * per + i];   // fixed order
        dst[i] = t;
    }
}

constexpr int PF_THREADS = 128;

// One CTA per output (l, shell): thread i sums the CTA slots i, i + 128, ...
// in order, then a fixed tree over the threads (the same order on every run).
__global__ void __launch_bounds__(PF_THREADS) k_power_final(const double* __restrict__ partial, int nblocks, int nsh,
                                                            int nell, double V, double nbar, double num_scale,
                                                            int nbatch, double* __restrict__ P,
                                                            double* __restrict__ Nk) {
    __shared__ double red[3][PF_THREADS];
    const int t = blockIdx.x;
    const int l = t / nsh, s = t % nsh, per = (2 * nell + 1) * nsh;
    double sp = 0.0, sw = 0.0, sn = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += PF_THREADS) {
        const double* q = partial + (size_t)b * per;
        sp += q[l * nsh + s];
        sw += q[(nell + l) * nsh + s];
        sn += q[2 * nell * nsh + s];
    }
    red[0][threadIdx.x] = sp;
    red[1][threadIdx.x] = sw;
    red[2][threadIdx.x] = sn;
    __syncthreads();
    for (int h = PF_THREADS / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h)
            for (int c = 0; c < 3; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    sp = red[0][0];
    sw = red[1][0];
    sn = red[2][0];
    double v = 0.0;
    if (sn > 0.0) {
        v = num_scale * sp / (V * sn);
        if (nbar > 0.0) v -= sw / (nbar * sn);
    }
    P[t] = v;
    if (Nk && l == 0) Nk[s] = sn / (double)nbatch;
}

}  // namespace

size_t power_partial_bytes(int nblocks, int nsh, int nell) {
    return (size_t)nblocks * (size_t)(2 * nell + 1) * (size_t)nsh * sizeof(double);
}

cudaError_t launch_power(const cx<float>* delta, const cx<float>* Q, double num_scale, const FftGeom& g,
                         const int16_t* shell_of, int nsh, const PowerEll& ells, double V, double nbar, int nblocks,
                         double* partial, double* P, double* Nk, cudaStream_t st, int nbatch, size_t bstride,
                         int dc_weight, int n2top) {
    const size_t smem = (size_t)PW_WARPS * (2 * ells.n + 1) * nsh * sizeof(double);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    const bool shot = nbar > 0.0;
    auto kern = shot ? k_power_partial<true> : k_power_partial<false>;
    static size_t set[2] = {0, 0};   // raised once per size and variant, never inside a graph capture
    cudaError_t e;
    if (smem > 48 * 1024 && smem > set[shot]) {
        if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return e;
        set[shot] = smem;
    }
    if (nbatch < 1 || nbatch > 65535 || (nbatch > 1 && Q)) return cudaErrorInvalidValue;
    kern<<<dim3(nblocks, nbatch), 32 * PW_WARPS, smem, st>>>(delta, Q, g, shell_of, nsh, ells, partial, bstride,
                                                             dc_weight, n2top);
    k_power_final<<<ells.n * nsh, PF_THREADS, 0, st>>>(partial, nblocks * nbatch, nsh, ells.n, V, nbar, num_scale,
                                                        nbatch, P, Nk);
    return cudaGetLastError();
}

}  // namespace bsp
