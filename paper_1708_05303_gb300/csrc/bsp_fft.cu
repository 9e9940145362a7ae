// bsp_fft.cu -- shell/Legendre filter fused into a pruned, batched inverse
// 3-D FFT (complex along x, complex along y, complex-to-real along z).
//
// Computes, for each requested field f (Sec. 3.1: the filtered real-space
// fields D^{(l)}_k(x) = int_k d^3q e^{iq.x} delta^{(l)}(q) under
// Eq. Standard_ell_Estim; Sec. 3.5: M^{(l)}_n(x) of Eq. betaEst),
//
//   F_f(x) = sum_n W_f(n) S_f(n) e^{+2 pi i n.x / N},
//   W_f(n) = w_l(mu) x {1[n in shell] | R_p[|n|^2]},  w_l = (2l+1) L_l,
//   S_f(n) = delta(n) | 1 | |delta(n)|^2,
//
// over the Hermitian half spectrum delta[N][N][N/2+1].  No 1/N^3 factor.
//
// Pruning: all weights vanish for |n| >= the last shell edge, so only
// frequencies |f| <= K on x and y and 0 <= f_z < nKz are carried:
//   pass 1: per (f_y, f_z) pencil, filter + inverse DFT along x
//           -> T1[f_y (compact)][x][f_z]
//   pass 2: per (x, f_z) pencil, inverse DFT along y -> T2[x][y][f_z]
//   pass 3: per (x, y) pencil, real inverse DFT along z -> F[x][y][z]
// Each pass stages a batch of pencils in shared memory, so global reads and
// writes are contiguous runs; the 1-D transforms are in-place Stockham
// autosort radix-2/3/4/5/8 stages, ping-ponging between two shared-memory
// buffers with one barrier per stage.  Twiddles come from a host table of
// exp(+2 pi i t/N) computed in FP64.
#include <algorithm>
#include <type_traits>

#include "bsp_internal.h"

namespace bsp {

namespace {

constexpr int NTHR = 256;

template <typename R>
__device__ __forceinline__ cx<R> cmul(cx<R> a, cx<R> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R>
__device__ __forceinline__ cx<R> cadd(cx<R> a, cx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R>
__device__ __forceinline__ cx<R> csub(cx<R> a, cx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <typename R>
__device__ __forceinline__ cx<R> cmuli(cx<R> a) { return {-a.im, a.re}; }   // i * a
template <typename R>
__device__ __forceinline__ cx<R> cscale(cx<R> a, R s) { return {a.re * s, a.im * s}; }

// Inverse (sign +1) DFT of RADIX values in registers: y_q = sum_r v_r e^{+2 pi i r q / RADIX}.
template <typename R, int RADIX>
__device__ __forceinline__ void butterfly(cx<R>* v) {
    if constexpr (RADIX == 2) {
        cx<R> a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if constexpr (RADIX == 4) {
        cx<R> s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
        cx<R> s13 = cadd(v[1], v[3]), d13 = cmuli(csub(v[1], v[3]));
        v[0] = cadd(s02, s13);
        v[2] = csub(s02, s13);
        v[1] = cadd(d02, d13);
        v[3] = csub(d02, d13);
    } else if constexpr (RADIX == 8) {
        cx<R> e[4] = {v[0], v[2], v[4], v[6]};
        cx<R> o[4] = {v[1], v[3], v[5], v[7]};
        butterfly<R, 4>(e);
        butterfly<R, 4>(o);
        const R h = (R)0.70710678118654752440;   // 1/sqrt(2)
        cx<R> w1o = {(o[1].re - o[1].im) * h, (o[1].re + o[1].im) * h};     // e^{i pi/4} o1
        cx<R> w2o = cmuli(o[2]);                                             // e^{i pi/2} o2
        cx<R> w3o = {-(o[3].re + o[3].im) * h, (o[3].re - o[3].im) * h};    // e^{3i pi/4} o3
        v[0] = cadd(e[0], o[0]);
        v[4] = csub(e[0], o[0]);
        v[1] = cadd(e[1], w1o);
        v[5] = csub(e[1], w1o);
        v[2] = cadd(e[2], w2o);
        v[6] = csub(e[2], w2o);
        v[3] = cadd(e[3], w3o);
        v[7] = csub(e[3], w3o);
    } else if constexpr (RADIX == 16) {
        // 16 = 4 x 4: X[k1 + 4 k2] = sum_j2 W4^{j2 k2} W16^{j2 k1} sum_j1 x[j2 + 4 j1] W4^{j1 k1}
        const R c1 = (R)0.92387953251128675613, s1 = (R)0.38268343236508977173;   // cos, sin 2pi/16
        const R h = (R)0.70710678118654752440;
        const cx<R> w[10] = {{(R)1, (R)0}, {c1, s1}, {h, h}, {s1, c1}, {(R)0, (R)1},
                             {-s1, c1}, {-h, h}, {-c1, s1}, {(R)-1, (R)0}, {-c1, -s1}};   // W16^m, m = 0..9
        cx<R> a[4][4];
#pragma unroll
        for (int j2 = 0; j2 < 4; ++j2) {
            cx<R> t[4] = {v[j2], v[j2 + 4], v[j2 + 8], v[j2 + 12]};
            butterfly<R, 4>(t);
#pragma unroll
            for (int k1 = 0; k1 < 4; ++k1) a[j2][k1] = (j2 * k1 == 0) ? t[k1] : cmul(t[k1], w[j2 * k1]);
        }
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            cx<R> u[4] = {a[0][k1], a[1][k1], a[2][k1], a[3][k1]};
            butterfly<R, 4>(u);
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = u[k2];
        }
    } else if constexpr (RADIX == 3) {
        const R s3 = (R)0.86602540378443864676;  // sqrt(3)/2
        cx<R> t = cadd(v[1], v[2]), d = csub(v[1], v[2]);
        cx<R> m = {v[0].re - (R)0.5 * t.re, v[0].im - (R)0.5 * t.im};
        cx<R> id = cmuli(cscale(d, s3));
        v[0] = cadd(v[0], t);
        v[1] = cadd(m, id);
        v[2] = csub(m, id);
    } else if constexpr (RADIX == 5) {
        const R c1 = (R)0.30901699437494742410, c2 = (R)-0.80901699437494742410;   // cos 2pi/5, cos 4pi/5
        const R s1 = (R)0.95105651629515357212, s2 = (R)0.58778525229247312917;    // sin 2pi/5, sin 4pi/5
        cx<R> t1 = cadd(v[1], v[4]), d1 = csub(v[1], v[4]);
        cx<R> t2 = cadd(v[2], v[3]), d2 = csub(v[2], v[3]);
        cx<R> a1 = {v[0].re + c1 * t1.re + c2 * t2.re, v[0].im + c1 * t1.im + c2 * t2.im};
        cx<R> a2 = {v[0].re + c2 * t1.re + c1 * t2.re, v[0].im + c2 * t1.im + c1 * t2.im};
        cx<R> b1 = cmuli(cx<R>{s1 * d1.re + s2 * d2.re, s1 * d1.im + s2 * d2.im});
        cx<R> b2 = cmuli(cx<R>{s2 * d1.re - s1 * d2.re, s2 * d1.im - s1 * d2.im});
        v[0] = cadd(v[0], cadd(t1, t2));
        v[1] = cadd(a1, b1);
        v[4] = csub(a1, b1);
        v[2] = cadd(a2, b2);
        v[3] = csub(a2, b2);
    }
}

// Shared-memory layouts of P pencils of length M (one element = one complex):
//   pencil-fast (passes 1, 2):  (p, i) -> i P + p + i/8
//   index-fast  (pass 3):       (p, i) -> p PS + i + i/8,  PS = M + M/8 + 1
// The i/8 padding spreads the strided Stockham accesses over all banks.
template <bool PF, int P>
__device__ __forceinline__ int sidx(int p, int i, int M) {
    return PF ? i * P + p + (i >> 3) : p * (M + (M >> 3) + 1) + i + (i >> 3);
}
template <bool PF, int P>
__host__ __device__ constexpr int smem_elems(int M) {
    return PF ? M * P + (M >> 3) + 1 : P * (M + (M >> 3) + 1);
}

// One Stockham stage of radix RADIX over P pencils of length M, out of
// place from src to dst.  Butterfly j reads x[j + r M/RADIX], twiddles by
// W_M^{r (j mod Ns) M/(Ns RADIX)} and writes y[(j/Ns) Ns RADIX + j mod Ns + r Ns]
// (autosort: natural order after the last stage).  With M and Ns compile-time
// constants (the specialised kernels) all index arithmetic folds to shifts.
template <typename R, int RADIX, bool PF, int P>
__device__ __forceinline__ void fft_stage(const cx<R>* __restrict__ src, cx<R>* __restrict__ dst, int M, int Ns,
                                          const cx<R>* tw, int twmul) {
    const int nbf = M / RADIX;
    const int total = nbf * P;
    for (int b = threadIdx.x; b < total; b += NTHR) {
        int p, j;
        if (PF) { p = b % P; j = b / P; } else { j = b % nbf; p = b / nbf; }
        const int k = j % Ns;
        const int tstep = k * (M / (Ns * RADIX)) * twmul;
        cx<R> v[RADIX];
#pragma unroll
        for (int r = 0; r < RADIX; ++r) {
            const cx<R> x = src[sidx<PF, P>(p, j + r * nbf, M)];
            v[r] = r == 0 ? x : cmul(x, tw[r * tstep]);
        }
        butterfly<R, RADIX>(v);
        const int o = (j / Ns) * Ns * RADIX + k;
#pragma unroll
        for (int r = 0; r < RADIX; ++r) dst[sidx<PF, P>(p, o + r * Ns, M)] = v[r];
    }
    __syncthreads();
}

// Runtime radix list (any supported length).  Returns the result buffer.
template <typename R, bool PF, int P>
__device__ cx<R>* fft_pingpong(cx<R>* a, cx<R>* b, int M, const int* rad, int nrad, const cx<R>* tw, int twmul) {
    int Ns = 1;
    for (int s = 0; s < nrad; ++s) {
        switch (rad[s]) {
            case 8: fft_stage<R, 8, PF, P>(a, b, M, Ns, tw, twmul); break;
            case 4: fft_stage<R, 4, PF, P>(a, b, M, Ns, tw, twmul); break;
            case 2: fft_stage<R, 2, PF, P>(a, b, M, Ns, tw, twmul); break;
            case 3: fft_stage<R, 3, PF, P>(a, b, M, Ns, tw, twmul); break;
            case 5: fft_stage<R, 5, PF, P>(a, b, M, Ns, tw, twmul); break;
        }
        Ns *= rad[s];
        cx<R>* t = a; a = b; b = t;
    }
    return a;
}

// Compile-time radix list: 16s for the power of two (with one 8 and/or 4 for
// the leftover; 2^9 = 16 x 8 x 4), then 3s and 5s.  The host's plan for the
// run-time kernels uses radices up to 8; both give the same transform.
struct RadixList {
    int n;
    int r[8];
};
__host__ __device__ constexpr RadixList radix_list(int m) {
    RadixList L{0, {0, 0, 0, 0, 0, 0, 0, 0}};
    int a = 0;
    while (m % 2 == 0) { m /= 2; ++a; }
    int n16 = a / 4, rem = a % 4;
    if (rem == 1 && n16 > 0) { --n16; }
    for (int i = 0; i < n16; ++i) L.r[L.n++] = 16;
    if (rem == 3) L.r[L.n++] = 8;
    else if (rem == 2) L.r[L.n++] = 4;
    else if (rem == 1 && a >= 5) { L.r[L.n++] = 8; L.r[L.n++] = 4; }
    else if (rem == 1) L.r[L.n++] = 2;
    while (m % 3 == 0) { m /= 3; L.r[L.n++] = 3; }
    while (m % 5 == 0) { m /= 5; L.r[L.n++] = 5; }
    return L;
}

template <typename R, bool PF, int P, int M, int S = 0, int NS = 1>
__device__ __forceinline__ cx<R>* fft_ct(cx<R>* a, cx<R>* b, const cx<R>* tw, int twmul) {
    constexpr RadixList L = radix_list(M);
    if constexpr (S >= L.n) {
        return a;
    } else {
        constexpr int RADIX = L.r[S];
        fft_stage<R, RADIX, PF, P>(a, b, M, NS, tw, twmul);
        return fft_ct<R, PF, P, M, S + 1, NS * RADIX>(b, a, tw, twmul);
    }
}

__device__ __forceinline__ int freq_of(int idx, int n) { return idx < n / 2 ? idx : idx - n; }

// Largest |frequency component| where the field can be nonzero (its shell's
// outer edge, at most K).  Every pass uses the same bound: pass 1 skips the
// pencils beyond it (f_y or f_z), pass 2 skips the f_z beyond it and reads no
// f_y beyond it, pass 3 reads no f_z beyond it, so nothing unwritten is read.
__device__ __forceinline__ int field_ext(const FieldDesc& fd, const FftGeom& g) {
    return fd.kext > 0 ? min(fd.kext, g.K) : g.K;
}

// W_f(n): the field's radial factor times w_l(mu), mu^2 = n_z^2/|n|^2.
template <typename R>
__device__ __forceinline__ R filter_weight(const FieldDesc& fd, int n2, int fz, const int16_t* shell_of,
                                           const float* radial, int n2max) {
    if (n2 <= 0 || n2 > n2max) return (R)0;
    R base;
    if (fd.kind == FIELD_RAW) return (R)1;
    if (fd.kind == FIELD_RADIAL) base = (R)radial[(size_t)fd.shell * (n2max + 1) + n2];
    else base = (shell_of[n2] == fd.shell) ? (R)1 : (R)0;
    if (base == (R)0 || fd.ell == 0) return base;
    const R mu2 = (R)(fz * fz) / (R)n2;
    if (fd.ell == 2) return base * (R)2.5 * ((R)3 * mu2 - (R)1);                       // 5 L_2
    return base * (R)1.125 * (((R)35 * mu2 - (R)30) * mu2 + (R)3);                     // 9 L_4
}

// Input of pass 1: the filtered spectrum W_f(n) S_f(n) at (f_x of ix, f_y of
// iy, k_z), zero outside the pruned range.
template <typename R>
__device__ __forceinline__ cx<R> pass1_input(const FftGeom& g, const FieldDesc& fd, const cx<float>* __restrict__ delta,
                                             const int16_t* __restrict__ shell_of, const float* __restrict__ radial,
                                             int N, int ix, int fy, int iy, int kz) {
    const int fx = freq_of(ix, N);
    cx<R> val = {(R)0, (R)0};
    if (kz < g.nKz && (!g.pruned || (fx >= -g.K && fx <= g.K))) {
        const int fz = (kz == N / 2) ? -(N / 2) : kz;
        const int n2 = fx * fx + fy * fy + fz * fz;
        const R w = filter_weight<R>(fd, n2, fz, shell_of, radial, g.n2max);
        if (w != (R)0) {
            if (fd.kind == FIELD_UNIT) {
                val.re = w;
            } else {
                const cx<float> d = delta[((size_t)ix * N + iy) * (N / 2 + 1) + kz];
                if (fd.kind == FIELD_POWER) {
                    // |delta|^2 of the Hermitian part: on the n_z = 0 and n/2 planes the
                    // half spectrum holds both n and -n, (delta(n) + conj delta(-n)) / 2
                    R re = (R)d.re, im = (R)d.im;
                    if (kz == 0 || kz == N / 2) {
                        const cx<float> m = delta[((size_t)((N - ix) % N) * N + (N - iy) % N) * (N / 2 + 1) + kz];
                        re = (R)0.5 * (re + (R)m.re);
                        im = (R)0.5 * (im - (R)m.im);
                    }
                    val.re = w * (re * re + im * im);
                } else {
                    val.re = w * (R)d.re;
                    val.im = w * (R)d.im;
                }
            }
        }
    }
    return val;
}

// Pass 1: filter + inverse DFT along x for P consecutive f_z of one f_y.
template <typename R, int P, int NN>
__global__ void __launch_bounds__(NTHR) k_pass1(FftGeom g, const cx<float>* __restrict__ delta,
                                                const int16_t* __restrict__ shell_of,
                                                const float* __restrict__ radial,
                                                const FieldDesc* __restrict__ fields,
                                                const cx<R>* __restrict__ twg, cx<R>* __restrict__ t1,
                                                size_t t1_stride) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = NN ? NN : g.n;
    cx<R>* tw = reinterpret_cast<cx<R>*>(smem_raw);
    cx<R>* buf = tw + N;
    cx<R>* scr = buf + smem_elems<true, P>(N);
    const FieldDesc fd = fields[blockIdx.y];
    const int nkzb = (g.nKz + P - 1) / P;
    const int cy = blockIdx.x / nkzb, kz0 = (blockIdx.x % nkzb) * P;
    const int fy = g.pruned ? cy - g.K : freq_of(cy, N);
    const int iy = (fy + N) % N;
    const int ke = field_ext(fd, g);
    if (fy > ke || fy < -ke || kz0 > ke) return;   // zero there, and pass 2 reads none of it
    for (int t = threadIdx.x; t < N; t += NTHR) tw[t] = twg[t];
    for (int e = threadIdx.x; e < N * P; e += NTHR) {
        const int p = e % P, ix = e / P, kz = kz0 + p;
        const cx<R> val = pass1_input<R>(g, fd, delta, shell_of, radial, N, ix, fy, iy, kz);
        buf[sidx<true, P>(p, ix, N)] = val;
    }
    __syncthreads();
    const cx<R>* res;
    if constexpr (NN > 0) res = fft_ct<R, true, P, NN>(buf, scr, tw, 1);
    else res = fft_pingpong<R, true, P>(buf, scr, N, g.rad, g.nrad, tw, 1);
    cx<R>* dst = t1 + (size_t)blockIdx.y * t1_stride;
    for (int e = threadIdx.x; e < N * P; e += NTHR) {
        const int p = e % P, x = e / P, kz = kz0 + p;
        if (kz < g.nKz) dst[((size_t)cy * N + x) * g.nKz + kz] = res[sidx<true, P>(p, x, N)];
    }
}

// Pass 2: inverse DFT along y for P consecutive f_z of one x.
__device__ __forceinline__ void block_max_to(unsigned* dst, float m) {
    // m >= 0: the float bit patterns order like the values
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(dst, __float_as_uint(m));
}

// Power of two s with bound * s in [2^(t-1), 2^t): t = 15 keeps 16-bit
// values below the FP16 maximum; t = 7 keeps a product of two scaled pair
// factors below 2^14.  Exact, so dividing by s afterwards is exact.
__device__ __forceinline__ float pow2_scale(float bound, int t = 15) {
    if (!(bound > 0.f)) return 1.f;
    int e;
    frexpf(bound, &e);
    return ldexpf(1.f, t - e);
}

template <typename R, int P, int NN>
__global__ void __launch_bounds__(NTHR) k_pass2(FftGeom g, const cx<R>* __restrict__ t1,
                                                size_t t1_stride, const cx<R>* __restrict__ twg,
                                                cx<R>* __restrict__ t2, size_t t2_stride,
                                                const FieldDesc* __restrict__ fields, unsigned* __restrict__ fmax2) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = NN ? NN : g.n;
    cx<R>* tw = reinterpret_cast<cx<R>*>(smem_raw);
    cx<R>* buf = tw + N;
    cx<R>* scr = buf + smem_elems<true, P>(N);
    const int nkzb = (g.nKz + P - 1) / P;
    const int x = blockIdx.x / nkzb, kz0 = (blockIdx.x % nkzb) * P;
    const int ke = field_ext(fields[blockIdx.y], g);
    if (kz0 > ke) return;   // zero there, and pass 3 reads none of it
    const cx<R>* src = t1 + (size_t)blockIdx.y * t1_stride;
    for (int t = threadIdx.x; t < N; t += NTHR) tw[t] = twg[t];
    for (int e = threadIdx.x; e < N * P; e += NTHR) {
        const int p = e % P, iy = e / P, kz = kz0 + p;
        const int fy = freq_of(iy, N);
        cx<R> val = {(R)0, (R)0};
        if (kz < g.nKz && fy >= -ke && fy <= ke) {
            const int cy = g.pruned ? fy + g.K : iy;
            val = src[((size_t)cy * N + x) * g.nKz + kz];
        }
        buf[sidx<true, P>(p, iy, N)] = val;
    }
    __syncthreads();
    const cx<R>* res;
    if constexpr (NN > 0) res = fft_ct<R, true, P, NN>(buf, scr, tw, 1);
    else res = fft_pingpong<R, true, P>(buf, scr, N, g.rad, g.nrad, tw, 1);
    cx<R>* dst = t2 + (size_t)blockIdx.y * t2_stride;
    float m = 0.f;
    for (int e = threadIdx.x; e < N * P; e += NTHR) {
        const int p = e % P, y = e / P, kz = kz0 + p;
        if (kz < g.nKz) {
            const cx<R> v = res[sidx<true, P>(p, y, N)];
            dst[((size_t)x * N + y) * g.nKz + kz] = v;
            m = fmaxf(m, (float)(fabs(v.re) + fabs(v.im)));
        }
    }
    if (fmax2) {
        const int f = fields[blockIdx.y].out16;
        if (f >= 0) block_max_to(fmax2 + f, m);
    }
}

// Pass 2 for n = 512 with the y-lines in registers: 8 lines (consecutive
// f_z of one x) per CTA, 32 threads per line, k_z fastest across the lanes so
// that every global load and store is a run of 8 consecutive f_z (64 bytes).
// With k = k1 + 32 k2 (thread k1 holds k2 = 0..15) and m = m1 + 16 m2,
//   z_m = sum_k1 W32^{k1 m2} [ W512^{k1 m1} sum_k2 X_{k1 + 32 k2} W16^{k2 m1} ],
// W_L = e^{2 pi i / L}; after one shared-memory transpose the outer 32-point
// DFT over k1 = j1 + 2 j2 is a 16-point DFT over j2 in each of two threads
// (j1 = 0, 1) and a radix-2 step between them through a shuffle:
//   z_{m1 + 16 (n + 16 q)} = U_0[n] + (-1)^q W32^n U_1[n].
constexpr int P2R = 8;
__host__ __device__ constexpr int p2r_idx(int row, int p) { return row * P2R + p + (row >> 4) * 8; }   // row = k1 * 16 + m1
constexpr size_t p2r_smem_bytes() { return sizeof(cx<float>) * (512 + (size_t)p2r_idx(511, P2R - 1) + 1); }

// The 512-point inverse DFT of the CTA's 8 lines.  On entry thread (k1 = 4 warp
// + c, line p) holds X_{k1 + 32 k2} in v[k2] and the twiddles are in tw; on
// return thread (m1 = 2 warp + (c >> 1), j1 = c & 1, line p) holds
// z_{m1 + 16 (n + 16 j1)} in v[n].  tr: the transpose buffer.
__device__ __forceinline__ void line512(cx<float> (&v)[16], const cx<float>* tw, cx<float>* tr, int warp, int c,
                                        int p) {
    const int k1 = 4 * warp + c;
    butterfly<float, 16>(v);   // v[m1] = sum_k2 X_{k1 + 32 k2} W16^{k2 m1}
#pragma unroll
    for (int m1 = 0; m1 < 16; ++m1) tr[p2r_idx(k1 * 16 + m1, p)] = m1 == 0 ? v[0] : cmul(v[m1], tw[k1 * m1]);
    __syncthreads();
    const int m1 = 2 * warp + (c >> 1), j1 = c & 1;
#pragma unroll
    for (int j2 = 0; j2 < 16; ++j2) v[j2] = tr[p2r_idx((j1 + 2 * j2) * 16 + m1, p)];
    butterfly<float, 16>(v);   // U_j1[n]
#pragma unroll
    for (int n = 0; n < 16; ++n) {
        cx<float> u = v[n];
        if (j1) u = cmul(u, tw[16 * n]);   // W32^n U_1[n]
        const cx<float> o = {__shfl_xor_sync(0xffffffffu, u.re, 8), __shfl_xor_sync(0xffffffffu, u.im, 8)};
        // j1 = 0 keeps U_0 + W U_1 (m2 = n), j1 = 1 keeps U_0 - W U_1 (m2 = n + 16)
        v[n] = j1 ? csub(o, u) : cadd(u, o);
    }
}

// Pass 1 for n = 512 with the x-lines in registers: 8 lines (consecutive
// f_z of one f_y) per CTA, laid out and transformed as in k_pass2r.
__global__ void __launch_bounds__(NTHR) k_pass1r(FftGeom g, const cx<float>* __restrict__ delta,
                                                 const int16_t* __restrict__ shell_of,
                                                 const float* __restrict__ radial,
                                                 const FieldDesc* __restrict__ fields,
                                                 const cx<float>* __restrict__ twg, cx<float>* __restrict__ t1,
                                                 size_t t1_stride) {
    constexpr int N = 512;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<float>* tw = reinterpret_cast<cx<float>*>(smem_raw);
    cx<float>* tr = tw + N;
    const FieldDesc fd = fields[blockIdx.y];
    const int nkzb = (g.nKz + P2R - 1) / P2R;
    const int cy = blockIdx.x / nkzb, kz0 = (blockIdx.x % nkzb) * P2R;
    const int fy = g.pruned ? cy - g.K : freq_of(cy, N);
    const int iy = (fy + N) % N;
    const int ke = field_ext(fd, g);
    if (fy > ke || fy < -ke || kz0 > ke) return;   // zero there, and pass 2 reads none of it
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int p = lane & 7, c = lane >> 3;
    const int kz = kz0 + p;
    for (int i = threadIdx.x; i < N; i += NTHR) tw[i] = twg[i];
    const int k1 = 4 * warp + c;
    cx<float> v[16];
#pragma unroll
    for (int k2 = 0; k2 < 16; ++k2) v[k2] = pass1_input<float>(g, fd, delta, shell_of, radial, N, k1 + 32 * k2, fy, iy, kz);
    __syncthreads();   // twiddles
    line512(v, tw, tr, warp, c, p);
    const int m1 = 2 * warp + (c >> 1), j1 = c & 1;
    if (kz < g.nKz) {
        cx<float>* dst = t1 + (size_t)blockIdx.y * t1_stride;
#pragma unroll
        for (int n = 0; n < 16; ++n) dst[((size_t)cy * N + m1 + 16 * (n + 16 * j1)) * g.nKz + kz] = v[n];
    }
}

__global__ void __launch_bounds__(NTHR) k_pass2r(FftGeom g, const cx<float>* __restrict__ t1, size_t t1_stride,
                                                 const cx<float>* __restrict__ twg, cx<float>* __restrict__ t2,
                                                 size_t t2_stride, const FieldDesc* __restrict__ fields,
                                                 unsigned* __restrict__ fmax2) {
    constexpr int N = 512;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<float>* tw = reinterpret_cast<cx<float>*>(smem_raw);
    cx<float>* tr = tw + N;
    const int nkzb = (g.nKz + P2R - 1) / P2R;
    const int x = blockIdx.x / nkzb, kz0 = (blockIdx.x % nkzb) * P2R;
    const int ke = field_ext(fields[blockIdx.y], g);
    if (kz0 > ke) return;   // zero there, and pass 3 reads none of it
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int p = lane & 7, c = lane >> 3;   // line (f_z offset) and lane group
    const int kz = kz0 + p;
    const bool live = kz < g.nKz;
    for (int i = threadIdx.x; i < N; i += NTHR) tw[i] = twg[i];
    const cx<float>* src = t1 + (size_t)blockIdx.y * t1_stride;
    // step A: thread k1 = 4 warp + c
    const int k1 = 4 * warp + c;
    cx<float> v[16];
#pragma unroll
    for (int k2 = 0; k2 < 16; ++k2) {
        const int iy = k1 + 32 * k2, fy = iy < N / 2 ? iy : iy - N;
        cx<float> val = {0.f, 0.f};
        if (live && fy >= -ke && fy <= ke) {
            const int cy = g.pruned ? fy + g.K : iy;
            val = src[((size_t)cy * N + x) * g.nKz + kz];
        }
        v[k2] = val;
    }
    __syncthreads();   // twiddles
    line512(v, tw, tr, warp, c, p);
    const int m1 = 2 * warp + (c >> 1), j1 = c & 1;
    cx<float>* dst = t2 + (size_t)blockIdx.y * t2_stride;
    float mx = 0.f;
#pragma unroll
    for (int n = 0; n < 16; ++n) {
        const int y = m1 + 16 * (n + 16 * j1);
        if (live) {
            dst[((size_t)x * N + y) * g.nKz + kz] = v[n];
            mx = fmaxf(mx, fabsf(v[n].re) + fabsf(v[n].im));
        }
    }
    if (fmax2) {
        const int f = fields[blockIdx.y].out16;
        if (f >= 0) block_max_to(fmax2 + f, mx);
    }
}

// Staging layouts of pass 3's z-lines in shared memory (element m of line p
// = F[2m] + i F[2m+1]).  Stockham passes: the i/8-padded index-fast layout.
template <int P>
struct StageStockham {
    __device__ static int idx(int p, int m, int M) { return sidx<false, P>(p, m, M); }
    template <typename R>
    __device__ static void load4(const cx<R>* res, int p, int m0, int M, cx<R> (&v)[4]) {
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i] = res[idx(p, m0 + i, M)];
    }
};
// Register pass 3 (M = 256): 16-element groups padded by 2 elements, lines
// 288 elements apart, so the 4 elements of a 16-byte output chunk are two
// aligned 16-byte loads and a quarter warp's loads fall on distinct banks.
struct Stage3r {
    static constexpr int PS = 288;
    __device__ static int idx(int p, int m, int) { return p * PS + m + (m >> 4) * 2; }
    template <typename R>
    __device__ static void load4(const cx<R>* res, int p, int m0, int, cx<R> (&v)[4]) {
        const float4* q = reinterpret_cast<const float4*>(res + idx(p, m0, 0));
        const float4 a = q[0], b = q[1];
        v[0] = {a.x, a.y};
        v[1] = {a.z, a.w};
        v[2] = {b.x, b.y};
        v[3] = {b.z, b.w};
    }
};

// Output of pass 3 for P consecutive y of one x: the real values of each
// z-line, res[sidx<false, P>(p, m, M)] = F[2m] + i F[2m+1], scaled and
// written as the field's FP32 row and/or 16-bit hi/lo planes.
template <typename R, int P, class Stage = StageStockham<P>>
__device__ __forceinline__ void pass3_store(const FftGeom& g, int N, int M, int x, int y0, const cx<R>* res,
                                            const FieldDesc& fd, R* __restrict__ out, size_t out_stride,
                                            uint32_t* __restrict__ hi, uint32_t* __restrict__ lo, int f16,
                                            const unsigned* __restrict__ fmax2, unsigned* __restrict__ f0max,
                                            FieldLayout lay) {
    const bool kbm = lay.groups16 > 0;
    R* dst = fd.out32 >= 0 ? out + (kbm ? (size_t)0 : (size_t)fd.out32 * out_stride) : nullptr;
    const size_t plane = (size_t)N * N * M;   // 32-bit words (two 16-bit values) per field plane
    uint32_t* dhi = nullptr;
    uint32_t* dlo = nullptr;
    if (fd.out16 >= 0 && hi) {
        if (kbm) {   // hi rows of the field's group, lo rows 1024 bytes further
            dhi = hi + (size_t)(fd.out16 >> 3) * 512 + (size_t)(fd.out16 & 7) * 32;
            dlo = lo ? dhi + 256 : nullptr;
        } else {
            dhi = hi + (size_t)fd.out16 * plane;
            dlo = lo ? lo + (size_t)fd.out16 * plane : nullptr;
        }
    }
    const int r32 = fd.out32 & 7, r16 = fd.out16 & 7;
    // |F(x,y,z)| <= sum_kz 2 |H_kz| <= 2 nKz max|T2|: the split planes are
    // scaled by the power of two that keeps that bound below 2^15
    const float bound = fmax2 && fd.out16 >= 0 ? 2.f * (float)g.nKz * __uint_as_float(fmax2[fd.out16]) : 0.f;
    const float sc = (dhi && fmax2) ? pow2_scale(bound) : 1.f;
    // FP32 pair factors of the tensor-core path are stored pre-scaled (|F s7| < 2^7)
    const R s7 = fmax2 ? (R)pow2_scale(bound, 7) : (R)1;
    float mx = 0.f;
    if constexpr (sizeof(R) == 4) {
        if (kbm && (M & 3) == 0) {
            // K-block-major output, four consecutive pairs of z per thread: one 16-byte
            // chunk of each 16-bit plane row and two of the FP32 row
            const int M4 = M >> 2;
            for (int e = threadIdx.x; e < M4 * P; e += NTHR) {
                const int m0 = (e % M4) * 4, p = e / M4, y = y0 + p;
                if (y >= N) continue;
                const size_t pos = ((size_t)x * N + y) * M + m0;
                const size_t kb = pos >> 5;
                const int w = (int)(pos & 31);   // a multiple of 4
                cx<R> v[4];
                Stage::load4(res, p, m0, M, v);
                if (dst) {
                    cx<R>* row = reinterpret_cast<cx<R>*>(dst) + (kb * (size_t)lay.rows32 + (size_t)fd.out32) * 32;
                    const int J = w >> 1;   // 16-byte chunks J, J + 1 of the 256-byte FP32 row
                    const int Ja = (J & 8) | ((J & 7) ^ r32), Jb = ((J + 1) & 8) | (((J + 1) & 7) ^ r32);
                    *reinterpret_cast<float4*>(row + 2 * Ja) =
                        make_float4(v[0].re * s7, v[0].im * s7, v[1].re * s7, v[1].im * s7);
                    *reinterpret_cast<float4*>(row + 2 * Jb) =
                        make_float4(v[2].re * s7, v[2].im * s7, v[3].re * s7, v[3].im * s7);
                    if (f0max)
#pragma unroll
                        for (int i = 0; i < 4; ++i) mx = fmaxf(mx, fmaxf(fabsf(v[i].re), fabsf(v[i].im)));
                }
                if (dhi) {
                    uint32_t h[4], l[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        // two consecutive z values -> 16-bit hi and lo (x0 in the low half)
                        const float x0 = v[i].re * sc, x1 = v[i].im * sc;
                        float h0, h1;
                        if (f16) {
                            asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(h[i]) : "f"(x1), "f"(x0));
                            unsigned short a = (unsigned short)(h[i] & 0xFFFFu), b = (unsigned short)(h[i] >> 16);
                            asm("cvt.f32.f16 %0, %1;" : "=f"(h0) : "h"(a));
                            asm("cvt.f32.f16 %0, %1;" : "=f"(h1) : "h"(b));
                            asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(l[i]) : "f"(x1 - h1), "f"(x0 - h0));
                        } else {
                            asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(h[i]) : "f"(x1), "f"(x0));
                            h0 = __uint_as_float(h[i] << 16);
                            h1 = __uint_as_float(h[i] & 0xFFFF0000u);
                            asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(l[i]) : "f"(x1 - h1), "f"(x0 - h0));
                        }
                    }
                    const size_t q = kb * (size_t)lay.groups16 * 512 + (size_t)(((w >> 2) ^ r16) << 2);
                    *reinterpret_cast<uint4*>(dhi + q) = make_uint4(h[0], h[1], h[2], h[3]);
                    if (dlo) *reinterpret_cast<uint4*>(dlo + q) = make_uint4(l[0], l[1], l[2], l[3]);
                }
            }
            if (f0max && dst) block_max_to(f0max + fd.out32, mx);
            return;
        }
    }
    for (int e = threadIdx.x; e < M * P; e += NTHR) {
        const int m = e % M, p = e / M, y = y0 + p;
        if (y >= N) continue;
        // pos counts pairs of consecutive z (one complex, one 32-bit plane word);
        // K-block-major: K-block pos / 32, pair w = pos % 32 of it (points 2w, 2w+1)
        const size_t pos = ((size_t)x * N + y) * M + m;
        size_t p32 = pos, p16 = pos;
        if (kbm) {
            const size_t kb = pos >> 5;
            const int w = (int)(pos & 31);
            const int J = w >> 1;   // 16-byte chunk of the 256-byte FP32 row
            p32 = (kb * (size_t)lay.rows32 + (size_t)fd.out32) * 32 + (size_t)(((J & 8) | ((J & 7) ^ r32)) * 2 + (w & 1));
            p16 = kb * (size_t)lay.groups16 * 512 + (size_t)((((w >> 2) ^ r16) << 2) | (w & 3));
        }
        const cx<R> v = res[Stage::idx(p, m, M)];
        if (dst) {
            reinterpret_cast<cx<R>*>(dst)[p32] = cx<R>{v.re * s7, v.im * s7};
            if (f0max) mx = fmaxf(mx, fmaxf(fabsf((float)v.re), fabsf((float)v.im)));
        }
        if (dhi) {
            // two consecutive z values -> 16-bit hi and lo planes (x0 in the low half)
            const float x0 = (float)v.re * sc, x1 = (float)v.im * sc;
            uint32_t h, l;
            if (f16) asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(h) : "f"(x1), "f"(x0));
            else asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(h) : "f"(x1), "f"(x0));
            float h0, h1;
            if (f16) {
                unsigned short a = (unsigned short)(h & 0xFFFFu), b = (unsigned short)(h >> 16);
                asm("cvt.f32.f16 %0, %1;" : "=f"(h0) : "h"(a));
                asm("cvt.f32.f16 %0, %1;" : "=f"(h1) : "h"(b));
            } else {
                h0 = __uint_as_float(h << 16);
                h1 = __uint_as_float(h & 0xFFFF0000u);
            }
            const float r0 = x0 - h0, r1 = x1 - h1;
            if (f16) asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(l) : "f"(r1), "f"(r0));
            else asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(l) : "f"(r1), "f"(r0));
            dhi[p16] = h;
            if (dlo) dlo[p16] = l;
        }
    }
    if (f0max && dst) block_max_to(f0max + fd.out32, mx);
}

// Pass 3: real inverse DFT along z for P consecutive y of one x, through a
// complex DFT of length M = N/2:  Z_k = (H_k + conj H_{M-k})
//   + i (H_k - conj H_{M-k}) e^{2 pi i k/N},  F[2m] = Re z_m, F[2m+1] = Im z_m,
// with Im H_0 = Im H_M = 0 (the Hermitian part of the n_z = 0, N/2 planes).
template <typename R, int P, int NN>
__global__ void __launch_bounds__(NTHR) k_pass3(FftGeom g, const cx<R>* __restrict__ t2,
                                                size_t t2_stride, const cx<R>* __restrict__ twg,
                                                const FieldDesc* __restrict__ fields, R* __restrict__ out,
                                                size_t out_stride, uint32_t* __restrict__ hi,
                                                uint32_t* __restrict__ lo, int f16,
                                                const unsigned* __restrict__ fmax2,
                                                unsigned* __restrict__ f0max, FieldLayout lay) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = NN ? NN : g.n, M = N / 2;
    cx<R>* tw = reinterpret_cast<cx<R>*>(smem_raw);
    cx<R>* buf = tw + N;
    cx<R>* scr = buf + smem_elems<false, P>(M);
    const int nyb = (N + P - 1) / P;
    const int x = blockIdx.x / nyb, y0 = (blockIdx.x % nyb) * P;
    const cx<R>* src = t2 + (size_t)blockIdx.y * t2_stride;
    const int nk = field_ext(fields[blockIdx.y], g) + 1;   // f_z read: 0 .. nk - 1
    for (int t = threadIdx.x; t < N; t += NTHR) tw[t] = twg[t];
    __syncthreads();
    for (int e = threadIdx.x; e < M * P; e += NTHR) {
        const int k = e % M, p = e / M, y = y0 + p;
        cx<R> z = {(R)0, (R)0};
        if (y < N) {
            const cx<R>* h = src + ((size_t)x * N + y) * g.nKz;
            cx<R> a = {(R)0, (R)0}, b = {(R)0, (R)0};
            if (k < nk) a = h[k];
            if (M - k < nk) b = h[M - k];
            if (k == 0) { a.im = (R)0; b.im = (R)0; }   // H_0 and H_M: real parts only
            const cx<R> bc = {b.re, -b.im};
            const cx<R> s = cadd(a, bc), d = csub(a, bc);
            z = cadd(s, cmuli(cmul(d, tw[k])));
        }
        buf[sidx<false, P>(p, k, M)] = z;
    }
    __syncthreads();
    const cx<R>* res;
    if constexpr (NN > 0) res = fft_ct<R, false, P, NN / 2>(buf, scr, tw, 2);
    else res = fft_pingpong<R, false, P>(buf, scr, M, g.rad_h, g.nrad_h, tw, 2);
    pass3_store<R, P>(g, N, M, x, y0, res, fields[blockIdx.y], out, out_stride, hi, lo, f16, fmax2, f0max, lay);
}

// Pass 3 for n = 512 (M = 256 = 16 x 16) with the z-lines in registers:
// 16 threads per line, P3R = 16 lines (consecutive y of one x) per CTA.
// With k = k1 + 16 k2 and m = m1 + 16 m2,
//   z_m = sum_k1 W16^{k1 m2} [ W256^{k1 m1} sum_k2 Z_{k1 + 16 k2} W16^{k2 m1} ],
// W_L = e^{2 pi i / L}: thread k1 forms its 16 inputs Z_{k1 + 16 k2} straight
// from T2 (the same Z_k as k_pass3), takes the inner 16-point DFT and the
// twiddle in registers, the lines pass once through shared memory
// (transposed), and thread m1 takes the outer 16-point DFT.  Two barriers
// instead of one per Stockham stage, and every thread busy in both DFTs.
constexpr int P3R = 16;
constexpr int P3R_TS = 16 * 17;   // transpose rows per line: 16 rows of 16 + 1 pad
constexpr int P3R_BUF = P3R * Stage3r::PS;   // staging buffer (the transpose fits in it)
constexpr size_t p3r_smem_bytes() { return sizeof(cx<float>) * (512 + 256 + (size_t)P3R_BUF); }
static_assert(P3R * P3R_TS <= P3R_BUF, "transpose fits in the output buffer");

__global__ void __launch_bounds__(NTHR) k_pass3r(FftGeom g, const cx<float>* __restrict__ t2, size_t t2_stride,
                                                 const cx<float>* __restrict__ twg,
                                                 const FieldDesc* __restrict__ fields, float* __restrict__ out,
                                                 size_t out_stride, uint32_t* __restrict__ hi,
                                                 uint32_t* __restrict__ lo, int f16,
                                                 const unsigned* __restrict__ fmax2,
                                                 unsigned* __restrict__ f0max, FieldLayout lay) {
    constexpr int N = 512, M = 256;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<float>* tw = reinterpret_cast<cx<float>*>(smem_raw);
    cx<float>* tw2 = tw + N;     // [m1][t] = W256^{t m1}: conflict-free reads across t
    cx<float>* buf = tw2 + 256;
    const int x = blockIdx.x / (N / P3R), y0 = (blockIdx.x % (N / P3R)) * P3R;
    const int p = threadIdx.x >> 4, t = threadIdx.x & 15;
    for (int i = threadIdx.x; i < N; i += NTHR) tw[i] = twg[i];
    tw2[threadIdx.x] = twg[(2 * (threadIdx.x & 15) * (threadIdx.x >> 4)) & (N - 1)];
    __syncthreads();
    const int nKz = g.nKz;
    const int nk = field_ext(fields[blockIdx.y], g) + 1;   // f_z read: 0 .. nk - 1
    const cx<float>* h = t2 + (size_t)blockIdx.y * t2_stride + ((size_t)x * N + y0 + p) * nKz;
    cx<float> v[16];
#pragma unroll
    for (int k2 = 0; k2 < 16; ++k2) {
        const int k = t + 16 * k2;
        cx<float> a = {0.f, 0.f}, b = {0.f, 0.f};
        if (k < nk) a = h[k];
        if (M - k < nk) b = h[M - k];
        if (k == 0) { a.im = 0.f; b.im = 0.f; }   // H_0 and H_M: real parts only
        const cx<float> bc = {b.re, -b.im};
        const cx<float> s = cadd(a, bc), d = csub(a, bc);
        v[k2] = cadd(s, cmuli(cmul(d, tw[k])));
    }
    butterfly<float, 16>(v);   // v[m1] = sum_k2 Z_{t + 16 k2} W16^{k2 m1}
    cx<float>* tr = buf + p * P3R_TS;
#pragma unroll
    for (int m1 = 0; m1 < 16; ++m1) tr[m1 * 17 + t] = m1 == 0 ? v[0] : cmul(v[m1], tw2[m1 * 16 + t]);   // W256^{t m1}
    __syncthreads();
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) v[k1] = tr[t * 17 + k1];
    butterfly<float, 16>(v);   // v[m2] = z_{t + 16 m2}
    __syncthreads();           // every line's transpose is read before the output layout reuses it
#pragma unroll
    for (int m2 = 0; m2 < 16; ++m2) buf[Stage3r::idx(p, t + 16 * m2, M)] = v[m2];
    __syncthreads();
    pass3_store<float, P3R, Stage3r>(g, N, M, x, y0, buf, fields[blockIdx.y], out, out_stride, hi, lo, f16, fmax2,
                                     f0max, lay);
}

template <typename R>
struct FftCfg;
template <>
struct FftCfg<float> {
    // pass-3 pencils are contiguous z-lines, so a smaller batch costs no
    // coalescing and lets more CTAs share an SM (about 39 KB each at n = 512)
    static constexpr int P = 8, P3 = 8;
};
template <>
struct FftCfg<double> {
    static constexpr int P = 4, P3 = 8;
};

template <typename R, int NN>
cudaError_t launch_n(const FftGeom& g, const cx<float>* delta, const int16_t* shell_of, const float* radial,
                     const FieldDesc* d_fields, int nfields, const cx<R>* tw, cx<R>* t1, cx<R>* t2, R* out,
                     size_t out_stride, uint32_t* hi, uint32_t* lo, int f16, unsigned* fmax2, unsigned* f0max,
                     cudaStream_t st, FieldLayout lay) {
    using C = FftCfg<R>;
    const int N = g.n, M = N / 2;
    const size_t t1_stride = (size_t)g.nK * N * g.nKz;
    const size_t t2_stride = (size_t)N * N * g.nKz;
    const size_t sm12 = sizeof(cx<R>) * ((size_t)N + 2 * (size_t)smem_elems<true, C::P>(N));
    const size_t sm3 = sizeof(cx<R>) * ((size_t)N + 2 * (size_t)smem_elems<false, C::P3>(M));
    // raise the dynamic shared-memory limit once per size (never inside a graph capture)
    static size_t set12 = 0, set3 = 0;
    cudaError_t e;
    if (sm12 > set12) {
        if ((e = cudaFuncSetAttribute(k_pass1<R, C::P, NN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)sm12)) != cudaSuccess)
            return e;
        if ((e = cudaFuncSetAttribute(k_pass2<R, C::P, NN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)sm12)) != cudaSuccess)
            return e;
        set12 = sm12;
    }
    if (sm3 > set3) {
        if ((e = cudaFuncSetAttribute(k_pass3<R, C::P3, NN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)sm3)) != cudaSuccess)
            return e;
        set3 = sm3;
    }
    const int nkzb = (g.nKz + C::P - 1) / C::P;
    dim3 g1(g.nK * nkzb, nfields), g2(N * nkzb, nfields), g3(N * ((N + C::P3 - 1) / C::P3), nfields);
    if constexpr (NN == 512 && std::is_same<R, float>::value) {
        static bool set1r = false;
        if (!set1r) {
            if ((e = cudaFuncSetAttribute(k_pass1r, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)p2r_smem_bytes())) != cudaSuccess)
                return e;
            set1r = true;
        }
        k_pass1r<<<dim3(g.nK * nkzb, nfields), NTHR, p2r_smem_bytes(), st>>>(g, delta, shell_of, radial, d_fields,
                                                                             tw, t1, t1_stride);
    } else {
        k_pass1<R, C::P, NN><<<g1, NTHR, sm12, st>>>(g, delta, shell_of, radial, d_fields, tw, t1, t1_stride);
    }
    if constexpr (NN == 512 && std::is_same<R, float>::value) {
        static bool set2r = false;
        if (!set2r) {
            if ((e = cudaFuncSetAttribute(k_pass2r, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)p2r_smem_bytes())) != cudaSuccess)
                return e;
            set2r = true;
        }
        k_pass2r<<<dim3(N * ((g.nKz + P2R - 1) / P2R), nfields), NTHR, p2r_smem_bytes(), st>>>(
            g, t1, t1_stride, tw, t2, t2_stride, d_fields, fmax2);
    } else {
        k_pass2<R, C::P, NN><<<g2, NTHR, sm12, st>>>(g, t1, t1_stride, tw, t2, t2_stride, d_fields, fmax2);
    }
    if constexpr (NN == 512 && std::is_same<R, float>::value) {
        static bool set3r = false;
        if (!set3r) {
            if ((e = cudaFuncSetAttribute(k_pass3r, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)p3r_smem_bytes())) != cudaSuccess)
                return e;
            set3r = true;
        }
        k_pass3r<<<dim3(N * (N / P3R), nfields), NTHR, p3r_smem_bytes(), st>>>(g, t2, t2_stride, tw, d_fields, out,
                                                                               out_stride, hi, lo, f16, fmax2,
                                                                               f0max, lay);
    } else {
        k_pass3<R, C::P3, NN><<<g3, NTHR, sm3, st>>>(g, t2, t2_stride, tw, d_fields, out, out_stride, hi, lo, f16,
                                                     fmax2, f0max, lay);
    }
    return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// Density input stage: cloud-in-cell with interlacing, then a forward
// real-to-complex 3-D FFT of both grids, combined into delta(k).  The
// forward transforms reuse the inverse Stockham stages through
// FFT(x) = conj(IFFT(conj x)).
// ---------------------------------------------------------------------------

// CIC weights of every particle on grid 1 (cells at j H) and grid 2 (cells at
// (j + 1/2) H): positions to cell units and fractions in FP64, weights added
// with FP32 atomics.
__global__ void k_cic(const float* __restrict__ pos, long long np, int n, double scale, float* __restrict__ g1,
                      float* __restrict__ g2) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < np;
         i += (long long)gridDim.x * blockDim.x) {
        const double p[3] = {(double)pos[3 * i], (double)pos[3 * i + 1], (double)pos[3 * i + 2]};
#pragma unroll
        for (int gs = 0; gs < 2; ++gs) {
            float* g = gs ? g2 : g1;
            int b[3];
            float t[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                double u = p[a] * scale - 0.5 * gs;
                u -= floor(u / n) * n;   // into [0, n)
                int bi = (int)floor(u);
                if (bi >= n) bi -= n;
                if (bi < 0) bi += n;
                b[a] = bi;
                t[a] = (float)(u - (double)bi);
            }
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int ox = (c >> 2) & 1, oy = (c >> 1) & 1, oz = c & 1;
                const float w = (ox ? t[0] : 1.f - t[0]) * (oy ? t[1] : 1.f - t[1]) * (oz ? t[2] : 1.f - t[2]);
                const int ix = (b[0] + ox) % n, iy = (b[1] + oy) % n, iz = (b[2] + oz) % n;
                atomicAdd(&g[((size_t)ix * n + iy) * n + iz], w);
            }
        }
    }
}

// exp(+2 pi i t / n), t < n, from FP64 sincospi.
__global__ void k_twiddles(int n, cx<float>* __restrict__ tw) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    double s, c;
    sincospi(2.0 * (double)t / (double)n, &s, &c);
    tw[t] = cx<float>{(float)c, (float)s};
}

// z pass: P real lines (x fixed, y0 .. y0 + P - 1) of grid blockIdx.y (or,
// with msub > 0, of the sub-cube blockIdx.y of side n of a grid of side
// nfull cut into msub^3 cubes), with
// delta = a g + b applied on load, packed as z_m = d_{2m} + i d_{2m+1}; an
// M = n/2-point FFT gives Z; X_k = E_k + e^{-2 pi i k/n} O_k with
// E_k = (Z_k + conj Z_{M-k})/2, O_k = (Z_k - conj Z_{M-k})/(2i), k = 0 .. M.
template <int P, int NN, bool SQ = false>
__global__ void __launch_bounds__(NTHR) k_fwd_z(FftGeom g, const float* __restrict__ grid, size_t gstride, float a,
                                                float b, const cx<float>* __restrict__ twg, cx<float>* __restrict__ T,
                                                size_t tstride, int msub = 0, int nfull = 0) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = NN ? NN : g.n, M = N / 2, H = M + 1;
    cx<float>* tw = reinterpret_cast<cx<float>*>(smem_raw);
    cx<float>* buf = tw + N;
    cx<float>* scr = buf + smem_elems<false, P>(M);
    const int nyb = (N + P - 1) / P;
    const int x = blockIdx.x / nyb, y0 = (blockIdx.x % nyb) * P;
    const float* src = grid + (size_t)blockIdx.y * gstride;
    size_t sx = (size_t)N * N, sy = (size_t)N;   // element strides of x and y in the source
    if (msub > 0) {
        const int c = blockIdx.y, cx_ = c / (msub * msub), cy = (c / msub) % msub, cz = c % msub;
        sx = (size_t)nfull * nfull;
        sy = (size_t)nfull;
        src = grid + (size_t)cx_ * N * sx + (size_t)cy * N * sy + (size_t)cz * N;
    }
    for (int t = threadIdx.x; t < N; t += NTHR) tw[t] = twg[t];
    for (int e = threadIdx.x; e < M * P; e += NTHR) {
        const int m = e % M, p = e / M, y = y0 + p;
        cx<float> v = {0.f, 0.f};
        if (y < N) {
            const float2 r = *reinterpret_cast<const float2*>(src + (size_t)x * sx + (size_t)y * sy + 2 * m);
            const float r0 = SQ ? r.x * r.x : r.x, r1 = SQ ? r.y * r.y : r.y;
            v = cx<float>{a * r0 + b, -(a * r1 + b)};   // conjugated
        }
        buf[sidx<false, P>(p, m, M)] = v;
    }
    __syncthreads();
    const cx<float>* res;
    if constexpr (NN > 0) res = fft_ct<float, false, P, NN / 2>(buf, scr, tw, 2);
    else res = fft_pingpong<float, false, P>(buf, scr, M, g.rad_h, g.nrad_h, tw, 2);
    cx<float>* dst = T + (size_t)blockIdx.y * tstride;
    for (int e = threadIdx.x; e < H * P; e += NTHR) {
        const int k = e % H, p = e / H, y = y0 + p;
        if (y >= N) continue;
        const cx<float> rk = res[sidx<false, P>(p, k % M, M)], rm = res[sidx<false, P>(p, (M - k) % M, M)];
        const cx<float> zk = {rk.re, -rk.im}, czm = {rm.re, rm.im};   // Z_k, conj Z_{M-k}
        const cx<float> E = cscale(cadd(zk, czm), 0.5f);
        const cx<float> D = cscale(csub(zk, czm), 0.5f);
        const cx<float> O = {D.im, -D.re};                               // D / i
        const cx<float> w = {tw[k].re, -tw[k].im};                       // e^{-2 pi i k/n}
        dst[((size_t)x * N + y) * H + k] = cadd(E, cmul(w, O));
    }
}

// y or x pass, in place: P consecutive k_z of one row o of grid blockIdx.y,
// element j at o * so + j * sj + k_z.
template <int P, int NN>
__global__ void __launch_bounds__(NTHR) k_fwd_axis(FftGeom g, const cx<float>* __restrict__ twg, cx<float>* T,
                                                   size_t tstride, size_t so, size_t sj) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = NN ? NN : g.n, H = N / 2 + 1;
    cx<float>* tw = reinterpret_cast<cx<float>*>(smem_raw);
    cx<float>* buf = tw + N;
    cx<float>* scr = buf + smem_elems<true, P>(N);
    const int nkzb = (H + P - 1) / P;
    const int o = blockIdx.x / nkzb, kz0 = (blockIdx.x % nkzb) * P;
    cx<float>* t = T + (size_t)blockIdx.y * tstride;
    for (int q = threadIdx.x; q < N; q += NTHR) tw[q] = twg[q];
    for (int e = threadIdx.x; e < N * P; e += NTHR) {
        const int p = e % P, j = e / P, kz = kz0 + p;
        cx<float> v = {0.f, 0.f};
        if (kz < H) {
            const cx<float> u = t[(size_t)o * so + (size_t)j * sj + kz];
            v = cx<float>{u.re, -u.im};
        }
        buf[sidx<true, P>(p, j, N)] = v;
    }
    __syncthreads();
    const cx<float>* res;
    if constexpr (NN > 0) res = fft_ct<float, true, P, NN>(buf, scr, tw, 1);
    else res = fft_pingpong<float, true, P>(buf, scr, N, g.rad, g.nrad, tw, 1);
    for (int e = threadIdx.x; e < N * P; e += NTHR) {
        const int p = e % P, j = e / P, kz = kz0 + p;
        if (kz < H) {
            const cx<float> r = res[sidx<true, P>(p, j, N)];
            t[(size_t)o * so + (size_t)j * sj + kz] = cx<float>{r.re, -r.im};
        }
    }
}

// delta(k) = (V/n^3) [X1(k) + e^{-i pi (n_x+n_y+n_z)/n} X2(k)] / (2 W(k)),
// W = prod_a sinc^2(pi n_a / n).
__global__ void k_fwd_combine(int N, const cx<float>* __restrict__ T1, const cx<float>* __restrict__ T2, float scale,
                              cx<float>* __restrict__ out) {
    const int H = N / 2 + 1;
    const size_t total = (size_t)N * N * H;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int kz = (int)(i % H), y = (int)((i / H) % N), x = (int)(i / ((size_t)H * N));
        const int fx = x < N / 2 ? x : x - N, fy = y < N / 2 ? y : y - N, fz = kz == N / 2 ? -(N / 2) : kz;
        float s, c;
        sincospif(-(float)(fx + fy + fz) / (float)N, &s, &c);
        float W = 1.f;
        const int f3[3] = {fx, fy, fz};
#pragma unroll
        for (int a = 0; a < 3; ++a)
            if (f3[a] != 0) {
                const float u = (float)f3[a] / (float)N;
                const float sc = sinpif(u) / (3.14159265358979f * u);
                W *= sc * sc;
            }
        const cx<float> a1 = T1[i], a2 = T2[i];
        const cx<float> ph = {c, s};
        out[i] = cscale(cadd(a1, cmul(ph, a2)), 0.5f * scale / W);
    }
}

template <int NN>
cudaError_t launch_density_n(const FftGeom& g, const float* pos, long long np, double box, char* ws,
                             cx<float>* out, cudaStream_t st) {
    constexpr int P = 8;
    const int N = g.n, M = N / 2, H = M + 1;
    const DensityLayout L = density_layout(N);
    cx<float>* tw = reinterpret_cast<cx<float>*>(ws + L.tw);
    float* grids = reinterpret_cast<float*>(ws + L.grids);
    cx<float>* T = reinterpret_cast<cx<float>*>(ws + L.spec);
    const size_t gstride = (size_t)N * N * N, tstride = (size_t)N * N * H;
    const size_t smz = sizeof(cx<float>) * ((size_t)N + 2 * (size_t)smem_elems<false, P>(M));
    const size_t sma = sizeof(cx<float>) * ((size_t)N + 2 * (size_t)smem_elems<true, P>(N));
    static size_t setz = 0, seta = 0;   // raised once per size, never inside a graph capture
    cudaError_t e;
    if (smz > setz) {
        if ((e = cudaFuncSetAttribute(k_fwd_z<P, NN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smz)) !=
            cudaSuccess)
            return e;
        setz = smz;
    }
    if (sma > seta) {
        if ((e = cudaFuncSetAttribute(k_fwd_axis<P, NN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sma)) !=
            cudaSuccess)
            return e;
        seta = sma;
    }
    if ((e = cudaMemsetAsync(grids, 0, 2 * gstride * sizeof(float), st)) != cudaSuccess) return e;
    k_twiddles<<<(N + 255) / 256, 256, 0, st>>>(N, tw);
    const int cic_blocks = (int)std::min<long long>(4096, (np + 255) / 256);
    k_cic<<<cic_blocks, 256, 0, st>>>(pos, np, N, (double)N / box, grids, grids + gstride);
    // delta_g = count / (N_p / n^3) - 1
    const float a = (float)((double)gstride / (double)np);
    k_fwd_z<P, NN><<<dim3(N * ((N + P - 1) / P), 2), NTHR, smz, st>>>(g, grids, gstride, a, -1.f, tw, T, tstride);
    const int nkzb = (H + P - 1) / P;
    k_fwd_axis<P, NN><<<dim3(N * nkzb, 2), NTHR, sma, st>>>(g, tw, T, tstride, (size_t)N * H, (size_t)H);   // along y
    k_fwd_axis<P, NN><<<dim3(N * nkzb, 2), NTHR, sma, st>>>(g, tw, T, tstride, (size_t)H, (size_t)N * H);   // along x
    const double V = box * box * box;
    k_fwd_combine<<<4096, 256, 0, st>>>(N, T, T + tstride, (float)(V / (double)gstride), out);
    return cudaGetLastError();
}
}  // namespace

// Sizes of the workloads get kernels specialised at compile time; any other
// supported size runs the same kernels with run-time radix lists.
template <typename R>
cudaError_t launch_fft_fields(const FftGeom& g, const cx<float>* delta, const int16_t* shell_of,
                              const float* radial, const FieldDesc* d_fields, int nfields,
                              const cx<R>* tw, cx<R>* t1, cx<R>* t2, R* out, size_t out_stride,
                              uint32_t* hi, uint32_t* lo, int f16, unsigned* fmax2, unsigned* f0max,
                              cudaStream_t st, FieldLayout lay) {
#define BSP_FFT_CASE(NV) \
    case NV:             \
        return launch_n<R, NV>(g, delta, shell_of, radial, d_fields, nfields, tw, t1, t2, out, out_stride, hi, lo, \
                               f16, fmax2, f0max, st, lay);
    switch (g.n) {
        BSP_FFT_CASE(64)
        BSP_FFT_CASE(96)
        BSP_FFT_CASE(128)
        BSP_FFT_CASE(160)
        BSP_FFT_CASE(256)
        BSP_FFT_CASE(512)
        default:
            return launch_n<R, 0>(g, delta, shell_of, radial, d_fields, nfields, tw, t1, t2, out, out_stride, hi, lo,
                                  f16, fmax2, f0max, st, lay);
    }
#undef BSP_FFT_CASE
}

template cudaError_t launch_fft_fields<float>(const FftGeom&, const cx<float>*, const int16_t*, const float*,
                                              const FieldDesc*, int, const cx<float>*, cx<float>*,
                                              cx<float>*, float*, size_t, uint32_t*, uint32_t*, int, unsigned*, unsigned*,
                                              cudaStream_t, FieldLayout);
DensityLayout density_layout(int n) {
    auto r256 = [](size_t b) { return (b + 255) / 256 * 256; };
    DensityLayout L{};
    const size_t n3 = (size_t)n * n * n, nh = (size_t)n * n * (n / 2 + 1);
    L.tw = 0;
    L.grids = r256(sizeof(cx<float>) * (size_t)n);
    L.spec = L.grids + r256(2 * n3 * sizeof(float));
    L.end = L.spec + r256(2 * nh * sizeof(cx<float>));
    return L;
}

template <int NN>
cudaError_t launch_forward_square_n(const FftGeom& g, const float* x, float a, const cx<float>* tw, cx<float>* T,
                                    cudaStream_t st) {
    constexpr int P = 8;
    const int N = g.n, M = N / 2, H = M + 1;
    const size_t smz = sizeof(cx<float>) * ((size_t)N + 2 * (size_t)smem_elems<false, P>(M));
    const size_t sma = sizeof(cx<float>) * ((size_t)N + 2 * (size_t)smem_elems<true, P>(N));
    static size_t setz = 0, seta = 0;   // raised once per size, never inside a graph capture
    cudaError_t e;
    if (smz > setz) {
        if ((e = cudaFuncSetAttribute(k_fwd_z<P, NN, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smz)) != cudaSuccess)
            return e;
        setz = smz;
    }
    if (sma > seta) {
        if ((e = cudaFuncSetAttribute(k_fwd_axis<P, NN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sma)) !=
            cudaSuccess)
            return e;
        seta = sma;
    }
    const size_t tstride = (size_t)N * N * H;
    k_fwd_z<P, NN, true><<<dim3(N * ((N + P - 1) / P), 1), NTHR, smz, st>>>(g, x, 0, a, 0.f, tw, T, tstride);
    const int nkzb = (H + P - 1) / P;
    k_fwd_axis<P, NN><<<dim3(N * nkzb, 1), NTHR, sma, st>>>(g, tw, T, tstride, (size_t)N * H, (size_t)H);
    k_fwd_axis<P, NN><<<dim3(N * nkzb, 1), NTHR, sma, st>>>(g, tw, T, tstride, (size_t)H, (size_t)N * H);
    return cudaGetLastError();
}

cudaError_t launch_forward_square(const FftGeom& g, const float* x, float a, const cx<float>* tw, cx<float>* T,
                                  cudaStream_t st) {
    switch (g.n) {
        case 64: return launch_forward_square_n<64>(g, x, a, tw, T, st);
        case 96: return launch_forward_square_n<96>(g, x, a, tw, T, st);
        case 128: return launch_forward_square_n<128>(g, x, a, tw, T, st);
        case 160: return launch_forward_square_n<160>(g, x, a, tw, T, st);
        case 256: return launch_forward_square_n<256>(g, x, a, tw, T, st);
        case 512: return launch_forward_square_n<512>(g, x, a, tw, T, st);
        default: return launch_forward_square_n<0>(g, x, a, tw, T, st);
    }
}

template <int NN>
cudaError_t launch_forward_subcubes_n(const FftGeom& g, int nfull, int m, const float* x, float a, cx<float>* tw,
                                      cx<float>* T, cudaStream_t st) {
    constexpr int P = 8;
    const int N = g.n, M = N / 2, H = M + 1, nc = m * m * m;
    const size_t smz = sizeof(cx<float>) * ((size_t)N + 2 * (size_t)smem_elems<false, P>(M));
    const size_t sma = sizeof(cx<float>) * ((size_t)N + 2 * (size_t)smem_elems<true, P>(N));
    static size_t setz = 0, seta = 0;   // raised once per size, never inside a graph capture
    cudaError_t e;
    if (smz > setz) {
        if ((e = cudaFuncSetAttribute(k_fwd_z<P, NN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smz)) !=
            cudaSuccess)
            return e;
        setz = smz;
    }
    if (sma > seta) {
        if ((e = cudaFuncSetAttribute(k_fwd_axis<P, NN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sma)) !=
            cudaSuccess)
            return e;
        seta = sma;
    }
    const size_t tstride = (size_t)N * N * H;
    k_twiddles<<<(N + 255) / 256, 256, 0, st>>>(N, tw);
    k_fwd_z<P, NN><<<dim3(N * ((N + P - 1) / P), nc), NTHR, smz, st>>>(g, x, 0, a, 0.f, tw, T, tstride, m, nfull);
    const int nkzb = (H + P - 1) / P;
    k_fwd_axis<P, NN><<<dim3(N * nkzb, nc), NTHR, sma, st>>>(g, tw, T, tstride, (size_t)N * H, (size_t)H);
    k_fwd_axis<P, NN><<<dim3(N * nkzb, nc), NTHR, sma, st>>>(g, tw, T, tstride, (size_t)H, (size_t)N * H);
    return cudaGetLastError();
}

cudaError_t launch_forward_subcubes(const FftGeom& g, int nfull, int m, const float* x, float a, cx<float>* tw,
                                    cx<float>* T, cudaStream_t st) {
    if (m < 1 || m * g.n != nfull || m * m * m > 65535) return cudaErrorInvalidValue;
    switch (g.n) {
        case 64: return launch_forward_subcubes_n<64>(g, nfull, m, x, a, tw, T, st);
        case 128: return launch_forward_subcubes_n<128>(g, nfull, m, x, a, tw, T, st);
        default: return launch_forward_subcubes_n<0>(g, nfull, m, x, a, tw, T, st);
    }
}

cudaError_t launch_density(const FftGeom& g, const float* pos, long long np, double box, void* ws,
                           cx<float>* out, cudaStream_t st) {
    char* w = reinterpret_cast<char*>(ws);
    switch (g.n) {
        case 64: return launch_density_n<64>(g, pos, np, box, w, out, st);
        case 96: return launch_density_n<96>(g, pos, np, box, w, out, st);
        case 128: return launch_density_n<128>(g, pos, np, box, w, out, st);
        case 160: return launch_density_n<160>(g, pos, np, box, w, out, st);
        case 256: return launch_density_n<256>(g, pos, np, box, w, out, st);
        case 512: return launch_density_n<512>(g, pos, np, box, w, out, st);
        default: return launch_density_n<0>(g, pos, np, box, w, out, st);
    }
}

template cudaError_t launch_fft_fields<double>(const FftGeom&, const cx<float>*, const int16_t*, const float*,
                                               const FieldDesc*, int, const cx<double>*, cx<double>*,
                                               cx<double>*, double*, size_t, uint32_t*, uint32_t*, int,
                                               unsigned*, unsigned*, cudaStream_t, FieldLayout);

}  // namespace bsp
