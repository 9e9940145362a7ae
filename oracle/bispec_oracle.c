/*
 * bispec_oracle.c -- plain FP64 CPU oracle for the FFT bispectrum-multipole
 * estimator of Regan, "An Inventory of Bispectrum Estimators for Redshift
 * Space Distortions" (arXiv:1708.05303).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA path and must never be reached from
 * the product path.
 *
 * What lives here (everything is FP64 and deliberately unoptimised):
 *   ora_fft1d       -- recursive mixed-radix DFT (any n; prime factors are
 *                      taken one at a time, a prime p by its O(p^2) DFT).
 *   ora_fft3d       -- 3-D DFT of a full complex grid, one axis at a time.
 *   ora_real_field  -- D(x) = sum_n W(n) delta(n) e^{+2 pi i n.x/N}, the
 *                      filtered real-space field of Sec. 3.1 (the
 *                      D_k^{(l)}(x) under Eq. "Standard_ell_Estim"), with
 *                      W the caller's shell x Legendre (or modal) weight.
 *   ora_sum3        -- sum_x A(x) B(x) C(x) per requested triple, Neumaier
 *                      compensated, plus sum_x (A B C)^2 for error scales
 *                      (the x-integral of Eq. "Standard_ell_Estim").
 *   ora_brute       -- the triangle sum itself, sum over n1, n2 with
 *                      n3 = -(n1+n2) mod N of W1 W2 W3 delta delta delta
 *                      (Eq. "Bisp_ell_restrict" aggregated over a bin),
 *                      for tiny grids.  It pins ora_real_field + ora_sum3.
 *
 * Parity pins for this file live in tests/test_oracle_pins.py.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef double complex cplx;

static int smallest_factor(int n) {
    for (int p = 2; (long)p * p <= n; p++)
        if (n % p == 0) return p;
    return n;
}

/* root[j] = exp(sign * 2 pi i j / n0), j = 0..n0-1 */
static cplx *make_roots(int n0, int sign) {
    cplx *r = (cplx *)malloc(sizeof(cplx) * (size_t)n0);
    if (!r) return NULL;
    for (int j = 0; j < n0; j++) {
        double ang = 2.0 * M_PI * (double)j / (double)n0;
        r[j] = cos(ang) + (double)sign * sin(ang) * I;
    }
    return r;
}

/*
 * out[k] = sum_{j<n} in[j*is] * exp(sign 2 pi i j k / n), out contiguous.
 * Decimation in time: with p the smallest factor of n and m = n/p,
 *   X[k0 + q m] = sum_r W_p^{r q} (W_n^{r k0} Y_r[k0]),
 * Y_r the length-m transform of the residue class j = r (mod p).
 * root[] holds the n0-th roots; W_n^t = root[(t * n0/n) mod n0].
 */
static void fft_rec(const cplx *in, long is, cplx *out, int n, const cplx *root,
                    int n0, cplx *tmp) {
    if (n == 1) {
        out[0] = in[0];
        return;
    }
    int p = smallest_factor(n), m = n / p;
    long step = n0 / n; /* W_n = root^step */
    for (int r = 0; r < p; r++) fft_rec(in + r * is, is * p, out + (long)r * m, m, root, n0, tmp);
    for (int k = 0; k < m; k++) {
        for (int r = 0; r < p; r++)
            tmp[r] = out[(long)r * m + k] * root[((long)r * k * step) % n0];
        for (int q = 0; q < p; q++) {
            cplx s = 0;
            for (int r = 0; r < p; r++) s += tmp[r] * root[((long)r * q * m * step) % n0];
            out[k + (long)q * m] = s;
        }
    }
}

/* In-place 1-D DFT of x[0..n) (stride 1), unnormalised; sign = -1 forward, +1 inverse. */
int ora_fft1d(cplx *x, int n, int sign) {
    if (n <= 0) return -1;
    cplx *root = make_roots(n, sign);
    cplx *buf = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    cplx *tmp = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    if (!root || !buf || !tmp) {
        free(root); free(buf); free(tmp);
        return -2;
    }
    fft_rec(x, 1, buf, n, root, n, tmp);
    memcpy(x, buf, sizeof(cplx) * (size_t)n);
    free(root); free(buf); free(tmp);
    return 0;
}

/* In-place 3-D DFT of a[n][n][n] (C order), unnormalised, one axis at a time. */
int ora_fft3d(cplx *a, int n, int sign) {
    if (n <= 0) return -1;
    cplx *root = make_roots(n, sign);
    if (!root) return -2;
    long n2 = (long)n * n;
    int status = 0;
    for (int axis = 0; axis < 3; axis++) {
        long stride = axis == 0 ? n2 : (axis == 1 ? n : 1);
#pragma omp parallel
        {
            cplx *line = (cplx *)malloc(sizeof(cplx) * (size_t)n);
            cplx *out = (cplx *)malloc(sizeof(cplx) * (size_t)n);
            cplx *tmp = (cplx *)malloc(sizeof(cplx) * (size_t)n);
            if (!line || !out || !tmp) {
#pragma omp atomic write
                status = -2;
            } else {
#pragma omp for schedule(static)
                for (long l = 0; l < n2; l++) {
                    /* the line's base: the two indices other than `axis` */
                    long u = l / n, v = l % n, base;
                    if (axis == 0) base = u * n + v;
                    else if (axis == 1) base = u * n2 + v;
                    else base = u * n2 + v * n;
                    for (int j = 0; j < n; j++) line[j] = a[base + j * stride];
                    fft_rec(line, 1, out, n, root, n, tmp);
                    for (int j = 0; j < n; j++) a[base + j * stride] = out[j];
                }
            }
            free(line); free(out); free(tmp);
        }
        if (status) break;
    }
    free(root);
    return status;
}

/*
 * F[x] = Re sum_n W[n] spec[n] exp(+2 pi i n.x / N) on the full grid
 * (spec, W: [N][N][N] in C order, n wrapped as 0..N-1).  The imaginary part
 * is discarded after measuring it: *max_imag = max_x |Im|, *max_real = max |Re|.
 */
int ora_real_field(const cplx *spec, const double *W, int n, double *F, double *max_imag,
                   double *max_real) {
    long n3 = (long)n * n * n;
    cplx *g = (cplx *)malloc(sizeof(cplx) * (size_t)n3);
    if (!g) return -2;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n3; i++) g[i] = W[i] * spec[i];
    int st = ora_fft3d(g, n, +1);
    if (st) {
        free(g);
        return st;
    }
    double mi = 0.0, mr = 0.0;
    for (long i = 0; i < n3; i++) {
        F[i] = creal(g[i]);
        double ai = fabs(cimag(g[i])), ar = fabs(F[i]);
        if (ai > mi) mi = ai;
        if (ar > mr) mr = ar;
    }
    *max_imag = mi;
    *max_real = mr;
    free(g);
    return 0;
}

/*
 * For each triple t: sums[t] = sum_x A(x) B(x) C(x), sumsq[t] = sum_x (A B C)^2,
 * with A = fields[tri[3t]], B = fields[tri[3t+1]], C = fields[tri[3t+2]].
 * Each triple is summed by one thread in x order with Neumaier compensation,
 * so results do not depend on the thread count.
 */
void ora_sum3(const double *const *fields, const int32_t *tri, long ntri, long npts, double *sums,
              double *sumsq) {
#pragma omp parallel for schedule(dynamic, 1)
    for (long t = 0; t < ntri; t++) {
        const double *A = fields[tri[3 * t]], *B = fields[tri[3 * t + 1]], *C = fields[tri[3 * t + 2]];
        double s = 0.0, comp = 0.0, q = 0.0, qc = 0.0;
        for (long x = 0; x < npts; x++) {
            double v = A[x] * B[x] * C[x];
            double u = s + v;
            if (fabs(s) >= fabs(v)) comp += (s - u) + v;
            else comp += (v - u) + s;
            s = u;
            double v2 = v * v, u2 = q + v2;
            if (q >= v2) qc += (q - u2) + v2;
            else qc += (v2 - u2) + q;
            q = u2;
        }
        sums[t] = s + comp;
        sumsq[t] = q + qc;
    }
}

/*
 * Direct triangle sum on a full grid [N][N][N]:
 *   S = sum_{i<n1, j<n2} W1[i] W2[j] W3[k] spec[i] spec[j] spec[k],
 *   k = flat index of -(n_i + n_j) mod N,
 * with i over the flat indices idx1[0..n1), j over idx2[0..n2) (the caller
 * passes the nonzero support of W1 and W2).  Also returns the unweighted,
 * spectrum-free count  sum 1[W1 != 0] 1[W2 != 0] 1[W3[k] != 0].
 */
void ora_brute(const cplx *spec, const double *W1, const double *W2, const double *W3, int n,
               const int64_t *idx1, long n1, const int64_t *idx2, long n2, double *out_re,
               double *out_im, double *count) {
    long nn = n;
    double sre = 0.0, sim = 0.0, cnt = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : sre, sim, cnt)
    for (long a = 0; a < n1; a++) {
        long i = idx1[a];
        long ix = i / (nn * nn), iy = (i / nn) % nn, iz = i % nn;
        cplx vi = W1[i] * spec[i];
        for (long b = 0; b < n2; b++) {
            long j = idx2[b];
            long jx = j / (nn * nn), jy = (j / nn) % nn, jz = j % nn;
            long kx = (2 * nn - ix - jx) % nn, ky = (2 * nn - iy - jy) % nn, kz = (2 * nn - iz - jz) % nn;
            long k = (kx * nn + ky) * nn + kz;
            if (W3[k] == 0.0) continue;
            cplx v = vi * (W2[j] * spec[j]) * (W3[k] * spec[k]);
            sre += creal(v);
            sim += cimag(v);
            cnt += 1.0;
        }
    }
    *out_re = sre;
    *out_im = sim;
    *count = cnt;
}

int ora_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
