// bsp_modal.cu -- host-side FP64 pieces of the modal estimator (Sec. 3.5):
// 1-D modes, radial filter tables, the ordering of 3-D modes, the inner-
// product matrix gamma over the tetrapyd, and the projection beta = gamma^-1 S.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/bsp.h"
#include "bsp_internal.h"

namespace bsp {

namespace {

// index of (a; b, c), b >= c, in the lexicographic list of all such triplets
__device__ __forceinline__ long long tri_index(int a, int b, int c, int nf) {
    return (long long)a * (nf * (nf + 1) / 2) + (long long)b * (b + 1) / 2 + c;
}

// <<B_l | Q_pqr>> for p <= q <= r from the raw sums (Sec. 3.5, Eq. Bisp_ell
// with the 1/6 permutation average):
//   l = 0: T0(r; q, p)
//   l = 2: T2(p; r, q) + T2(q; r, p) + T2(r; q, p)
//   l = 4: the same with T4, plus U(r; q, p) + U(p; r, q) + U(q; r, p),
// T^l(a; b, c) = sum_x M^l_a M0_b M0_c, U(a; b, c) = sum_x M0_a M2_b M2_c,
// all divided by n^3 V^3 (the x-integral and the three 1/V of M).
__global__ void k_modal_assemble(const double* __restrict__ T, const double* __restrict__ U,
                                 const int* __restrict__ ells, int n_ell, int nf, long long nall,
                                 int ntrip, double scale, double* __restrict__ S) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)n_ell * ntrip) return;
    const int li = (int)(i / ntrip);
    int t = (int)(i % ntrip);
    // unrank t -> (p <= q <= r) in lexicographic order
    int p = 0, q = 0, r = 0;
    for (p = 0; p < nf; ++p) {
        const int m = nf - p;   // pairs (q, r) with p <= q <= r < nf
        const int cnt = m * (m + 1) / 2;
        if (t < cnt) break;
        t -= cnt;
    }
    for (q = p; q < nf; ++q) {
        const int cnt = nf - q;
        if (t < cnt) break;
        t -= cnt;
    }
    r = q + t;
    const double* Tl = T + (long long)li * nall;
    double v;
    if (ells[li] == 0) {
        v = Tl[tri_index(r, q, p, nf)];
    } else {
        v = Tl[tri_index(p, r, q, nf)] + Tl[tri_index(q, r, p, nf)] + Tl[tri_index(r, q, p, nf)];
        if (ells[li] == 4 && U)
            v += U[tri_index(r, q, p, nf)] + U[tri_index(p, r, q, nf)] + U[tri_index(q, r, p, nf)];
    }
    S[i] = v * scale;
}

}  // namespace

cudaError_t launch_modal_assemble(const double* T, const double* U, const int* ells, int n_ell, int nf,
                                  long long nall, int ntrip, double scale, double* S, cudaStream_t st) {
    const long long n = (long long)n_ell * ntrip;
    if (n <= 0) return cudaSuccess;
    k_modal_assemble<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(T, U, ells, n_ell, nf, nall, ntrip, scale, S);
    return cudaGetLastError();
}

}  // namespace bsp

namespace {

// q_p(k): shifted Legendre polynomial P_p on [kmin, kmax], zero outside
// (Bonnet recurrence (j+1) P_{j+1} = (2j+1) t P_j - j P_{j-1}).
double qmode(int p, double k, double kmin, double kmax) {
    if (k < kmin || k > kmax) return 0.0;
    const double t = 2.0 * (k - kmin) / (kmax - kmin) - 1.0;
    double a = 1.0, b = t;
    if (p == 0) return a;
    for (int j = 1; j < p; ++j) {
        const double c = ((2 * j + 1) * t * b - j * a) / (j + 1);
        a = b;
        b = c;
    }
    return b;
}

// Gauss-Legendre nodes / weights on [-1, 1] by Newton iteration on P_n.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int j = 1; j < n; ++j) {
                const double p2 = ((2 * j + 1) * z * p1 - j * p0) / (j + 1);
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

}  // namespace

extern "C" {

bsp_status bsp_modal_radial_powerlaw(int n, double box, int n_modes, double kmin, double kmax, double amp,
                                     double n_s, int sqrt_k, double* table) {
    if (n < 8 || n % 2 || !(box > 0) || n_modes < 1 || n_modes > 64 || !(kmin >= 0) || !(kmax > kmin) ||
        !(amp > 0) || !table)
        return BSP_EINVAL;
    const int n2max = 3 * (n / 2) * (n / 2);
    const double kf = 2.0 * M_PI / box;
    for (int p = 0; p < n_modes; ++p)
        for (int n2 = 0; n2 <= n2max; ++n2) {
            double v = 0.0;
            if (n2 > 0) {
                const double k = kf * std::sqrt((double)n2);
                const double P = amp * std::pow(k, n_s);
                const double den = sqrt_k ? std::sqrt(k * P) : std::sqrt(P);
                v = qmode(p, k, kmin, kmax) / den;
                if (!std::isfinite(v)) v = 0.0;
            }
            table[(size_t)p * (n2max + 1) + n2] = v;
        }
    return BSP_OK;
}

bsp_status bsp_modal_modes(int n_modes_1d, int n_keep, int32_t* modes) {
    if (n_modes_1d < 1 || n_keep < 1 || !modes) return BSP_EINVAL;
    // all p <= q <= r, ordered by (p+q+r, p, q, r)
    int k = 0;
    for (int s = 0; s <= 3 * (n_modes_1d - 1) && k < n_keep; ++s)
        for (int p = 0; p < n_modes_1d && k < n_keep; ++p)
            for (int q = p; q < n_modes_1d && k < n_keep; ++q) {
                const int r = s - p - q;
                if (r < q || r >= n_modes_1d) continue;
                modes[3 * k] = p;
                modes[3 * k + 1] = q;
                modes[3 * k + 2] = r;
                ++k;
            }
    return k == n_keep ? BSP_OK : BSP_EINVAL;
}

bsp_status bsp_modal_gamma(int n_keep, const int32_t* modes, double kmin, double kmax, int npts, double* gamma) {
    if (n_keep < 1 || !modes || !(kmax > kmin) || !(kmin >= 0) || npts < 2 || npts > 256 || !gamma)
        return BSP_EINVAL;
    int pmax = 0;
    for (int i = 0; i < 3 * n_keep; ++i) {
        if (modes[i] < 0) return BSP_EINVAL;
        pmax = std::max(pmax, modes[i] + 1);
    }
    std::vector<double> gx, gw;
    gauss_legendre(npts, gx, gw);
    const double a = kmin, b = kmax;
    // The tetrapyd {k_i in [a, b], each k_i <= the sum of the other two}:
    // k1 over [max(a, |k2-k3|), min(b, k2+k3)]; the k3 integrand kinks where
    // those limits switch (k3 = b - k2, k2 - a, k2 + a) and the k2 one where
    // the kinks cross, so Gauss-Legendre on each piece is exact for the
    // polynomial integrand once npts is large enough.
    std::vector<double> cuts2 = {a, b};
    for (double v : {(a + b) / 2, (b - a) / 2, 2 * a, b - a})
        if (v > a && v < b) cuts2.push_back(v);
    std::sort(cuts2.begin(), cuts2.end());
    std::vector<double> G((size_t)n_keep * n_keep, 0.0);
    std::vector<double> q1(pmax), q2(pmax), q3(pmax), Q(n_keep);
    for (size_t i2 = 0; i2 + 1 < cuts2.size(); ++i2) {
        const double lo2 = cuts2[i2], hi2 = cuts2[i2 + 1];
        if (hi2 <= lo2) continue;
        for (int m2 = 0; m2 < npts; ++m2) {
            const double k2 = 0.5 * (hi2 - lo2) * gx[m2] + 0.5 * (hi2 + lo2);
            const double w2 = 0.5 * (hi2 - lo2) * gw[m2];
            std::vector<double> cuts3 = {a, b};
            for (double v : {b - k2, k2 - a, k2 + a})
                if (v > a && v < b) cuts3.push_back(v);
            std::sort(cuts3.begin(), cuts3.end());
            for (int p = 0; p < pmax; ++p) q2[p] = qmode(p, k2, a, b);
            for (size_t i3 = 0; i3 + 1 < cuts3.size(); ++i3) {
                const double lo3 = cuts3[i3], hi3 = cuts3[i3 + 1];
                if (hi3 <= lo3) continue;
                for (int m3 = 0; m3 < npts; ++m3) {
                    const double k3 = 0.5 * (hi3 - lo3) * gx[m3] + 0.5 * (hi3 + lo3);
                    const double w3 = 0.5 * (hi3 - lo3) * gw[m3];
                    const double lo1 = std::max(a, std::fabs(k2 - k3)), hi1 = std::min(b, k2 + k3);
                    if (hi1 <= lo1) continue;
                    for (int p = 0; p < pmax; ++p) q3[p] = qmode(p, k3, a, b);
                    for (int m1 = 0; m1 < npts; ++m1) {
                        const double k1 = 0.5 * (hi1 - lo1) * gx[m1] + 0.5 * (hi1 + lo1);
                        const double wt = 0.5 * (hi1 - lo1) * gw[m1] * w2 * w3;
                        for (int p = 0; p < pmax; ++p) q1[p] = qmode(p, k1, a, b);
                        // Q_n: the product q_p q_q q_r averaged over the 6 orderings of (k1, k2, k3)
                        for (int n = 0; n < n_keep; ++n) {
                            const int p = modes[3 * n], q = modes[3 * n + 1], r = modes[3 * n + 2];
                            Q[n] = (q1[p] * q2[q] * q3[r] + q1[p] * q2[r] * q3[q] + q1[q] * q2[p] * q3[r] +
                                    q1[q] * q2[r] * q3[p] + q1[r] * q2[p] * q3[q] + q1[r] * q2[q] * q3[p]) /
                                   6.0;
                        }
                        for (int n = 0; n < n_keep; ++n)
                            for (int m = 0; m <= n; ++m) G[(size_t)n * n_keep + m] += wt * Q[n] * Q[m];
                    }
                }
            }
        }
    }
    const double c = 1.0 / (8.0 * M_PI * M_PI * M_PI * M_PI);
    for (int n = 0; n < n_keep; ++n)
        for (int m = 0; m <= n; ++m) gamma[(size_t)n * n_keep + m] = gamma[(size_t)m * n_keep + n] =
            c * G[(size_t)n * n_keep + m];
    return BSP_OK;
}

bsp_status bsp_modal_project(int n_keep, const double* gamma, int n_rhs, const double* S, double* beta) {
    if (n_keep < 1 || !gamma || n_rhs < 1 || !S || !beta) return BSP_EINVAL;
    // Cholesky gamma = L L^T, then L y = s, L^T beta = y, per right-hand side
    std::vector<double> L((size_t)n_keep * n_keep, 0.0);
    for (int i = 0; i < n_keep; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = gamma[(size_t)i * n_keep + j];
            for (int k = 0; k < j; ++k) s -= L[(size_t)i * n_keep + k] * L[(size_t)j * n_keep + k];
            if (i == j) {
                if (!(s > 0)) return BSP_EINVAL;   // not positive definite
                L[(size_t)i * n_keep + i] = std::sqrt(s);
            } else {
                L[(size_t)i * n_keep + j] = s / L[(size_t)j * n_keep + j];
            }
        }
    std::vector<double> y(n_keep);
    for (int r = 0; r < n_rhs; ++r) {
        const double* s = S + (size_t)r * n_keep;
        double* x = beta + (size_t)r * n_keep;
        for (int i = 0; i < n_keep; ++i) {
            double v = s[i];
            for (int k = 0; k < i; ++k) v -= L[(size_t)i * n_keep + k] * y[k];
            y[i] = v / L[(size_t)i * n_keep + i];
        }
        for (int i = n_keep - 1; i >= 0; --i) {
            double v = y[i];
            for (int k = i + 1; k < n_keep; ++k) v -= L[(size_t)k * n_keep + i] * x[k];
            x[i] = v / L[(size_t)i * n_keep + i];
        }
    }
    return BSP_OK;
}

}  // extern "C"
