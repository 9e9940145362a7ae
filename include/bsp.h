/*
 * bsp.h -- C ABI of libbsp, a GB300 (sm_103a) implementation of the FFT
 * bispectrum-multipole estimator and its modal variant from Regan,
 * "An Inventory of Bispectrum Estimators for Redshift Space Distortions"
 * (arXiv:1708.05303).
 *
 * Problem statement (Sec. 3.1, Eq. Standard_ell_Estim and
 * Eq. Bisp_ell_restrict): given a gridded redshift-space density delta(k)
 * in a periodic box of volume V, k-shells [k +- dk/2] and even multipoles
 * l, return for every triangle bin (a, b, c), a >= b >= c,
 *
 *   B^l_abc = sum_{q1 in a, q2 in b, q3 in c, q1+q2+q3 = 0}
 *             w_l(mu_1) delta(q1) delta(q2) delta(q3) / (V N_abc),
 *
 * w_l(mu) = (2l+1) L_l(mu), mu_1 the cosine between q1 and the line of
 * sight z, N_abc the number of grid triangles in the bin (V_B of Sec. 3.1).
 * The Legendre leg is the largest shell a.  The sums are evaluated as
 * sum_x F^l_a(x) F^0_b(x) F^0_c(x) over real-space filtered fields
 * F^l_a(x) = sum_{n in a} w_l(mu) delta(n) e^{i k.x} produced by inverse
 * 3-D FFTs ("reduced to ... products of FFTs", Sec. 3.1).
 *
 * Conventions.
 *   - Grid: n^3, C order (x, y, z); z (the last axis) is the line of sight.
 *     Index j along an axis is frequency j for j < n/2, j - n otherwise.
 *   - delta(k) is the continuum-normalised half spectrum
 *     delta(k) = (V/n^3) sum_x delta_x e^{-i k.x}, complex64 [n][n][n/2+1],
 *     interleaved (re, im) float pairs.  On the n_z = 0 and n_z = n/2 planes
 *     only the Hermitian part is used (as a real inverse FFT does).
 *   - Shell a holds modes with edges[a]^2 <= |n|^2 < edges[a+1]^2, edges in
 *     units of k_f = 2 pi / L, ascending.
 *   - Bins: (a, b, c) with a >= b >= c, lexicographic, holding >= 1 triangle.
 *
 * Memory and ownership.
 *   - The caller owns every device buffer passed in (inputs, outputs and the
 *     workspace); sizes come from bsp_workspace_size.  Device pointers must
 *     be 256-byte aligned.
 *   - The plan owns small device tables (shell lookup, tile lists, counts)
 *     that it allocates at creation / bsp_counts and frees on destroy.
 *   - All GPU work is enqueued on the caller's stream (a cudaStream_t passed
 *     as void*; NULL = legacy default stream).  bsp_counts and
 *     bsp_compute_host synchronise that stream; bsp_compute does not.
 *
 * Errors.  Every entry point returns a bsp_status.  Argument errors are
 * detected before anything is enqueued and leave the plan unchanged.
 * CUDA errors map to BSP_ECUDA (the CUDA error string is available from
 * bsp_last_error).  No entry point aborts, traps or exits.
 */
#ifndef BSP_H
#define BSP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BSP_OK = 0,
    BSP_EINVAL = -1,        /* bad argument (null, size, order, alignment) */
    BSP_ENOMEM = -2,        /* a plan-owned allocation failed */
    BSP_ECUDA = -3,         /* a CUDA call or launch failed */
    BSP_EUNSUPPORTED = -4,  /* valid request this build does not support */
    BSP_ETIMEOUT = -5,      /* a bounded device wait gave up */
    BSP_ESTATE = -6         /* call out of order (e.g. compute before counts) */
} bsp_status;

/* Arithmetic of the contraction (the x-sum).  Fields, counts, reductions and
 * normalisation are FP32/FP64 whatever the choice. */
typedef enum {
    BSP_FP32 = 0,        /* CUDA-core FP32 FMA, FP32 partials flushed to FP64 */
    BSP_SPLIT_BF16 = 1,  /* tcgen05 BF16 hi+lo split products, FP32 accumulate */
    BSP_BF16 = 2,        /* tcgen05 BF16 hi only (reported, not gated) */
    BSP_SPLIT_F16 = 3    /* tcgen05 FP16 hi+lo split products of power-of-two scaled
                            operands (22 significant bits), FP32 accumulate */
} bsp_precision;

/* Plan flags. */
enum {
    BSP_SHOT_NOISE = 1u,  /* reserve workspace for Poisson shot-noise subtraction (BSP_FP32 only) */
    BSP_FULL_TENSOR = 2u  /* output T^l[a; b >= c] for every a, not only the largest shell (see below) */
};

typedef struct bsp_plan bsp_plan;

/*
 * Create a plan for the standard estimator (Sec. 3.1).
 *   n        grid side, even, 8 <= n <= 512, of the form 2^a 3^b 5^c.
 *   box      box side L (> 0); V = L^3.
 *   n_shells number of shells (1..64); edges_kf has n_shells+1 ascending
 *            values > 0 in units of k_f, the last <= sqrt(3) n / 2.
 *   n_ell    1..3 entries of ells, each in {0, 2, 4}, strictly ascending
 *            (odd l vanish by parity, Sec. 3.5).
 *   prec     a bsp_precision.
 *   flags    0, BSP_SHOT_NOISE (triples the field workspace; BSP_FP32 only),
 *            BSP_FULL_TENSOR, or both.
 * The paper puts the Legendre weight on the largest side (Sec. 3.1, "with
 * respect to the largest side"), so by default the bins are (a, b, c) with
 * a >= b >= c and the weight on a.  With BSP_FULL_TENSOR the output bins are
 * every distinct (a; b, c), b >= c, whose three shells form a valid bin, with
 * the weight on a whichever shell it is: a < b puts L_l on a smaller side,
 * so conventions that weight another leg (e.g. the first index of
 * T^l[i, j, k]) can be read off.  For l = 0 the extra entries repeat the
 * sorted bin's value.  Counts are those of the sorted bin.
 * Host-only: allocates the plan's small device tables on the current device.
 */
bsp_status bsp_plan_create(bsp_plan** out, int n, double box, int n_shells,
                           const double* edges_kf, int n_ell, const int* ells,
                           int prec, unsigned flags);

/*
 * Create a plan for the modal estimator (Sec. 3.5, Eq. betaEst and its RSD
 * form): fields M^l_p(x) = sum_n e^{ik.x} w_l(mu) R_p[|n|^2] delta(n), one
 * per 1-D mode p and multipole, and the raw projections
 *   <<B_l | Q_pqr>> = (1/(n^3 V^3)) sum_x sum_{l1+l2+l3=l} {M^(l1) M^(l2) M^(l3)}_pqr
 * for every p <= q <= r (the {} average over the 6 orderings of (p, q, r);
 * l = 2 needs 3 terms, l = 4 six, l = 0 one -- Eq. Bisp_ell and its footnote).
 *   n_funcs  1-D modes (1..64).
 *   radial   HOST FP64 [n_funcs][3 (n/2)^2 + 1]: R_p indexed by the integer
 *            |n|^2, e.g. q_p(k)/sqrt(k P(k)) from bsp_modal_radial_powerlaw.
 *            Copied (as FP32) into the plan.
 *   ells, prec as for bsp_plan_create; flags 0.
 * No counts are needed; bsp_counts and bsp_compute reject modal plans.
 */
bsp_status bsp_plan_create_modal(bsp_plan** out, int n, double box, int n_funcs, const double* radial,
                                 int n_ell, const int* ells, int prec, unsigned flags);

/* n_funcs and the number of triplets p <= q <= r, n_funcs (n_funcs+1)(n_funcs+2)/6. */
bsp_status bsp_modal_size(const bsp_plan* plan, int* n_funcs, int* n_trip);

/*
 * Raw modal projections <<B_l | Q_pqr>> (see bsp_plan_create_modal) into
 * S, device FP64 [n_ell][n_trip], triplets (p <= q <= r) in lexicographic
 * order.  delta_k and ws as for bsp_compute.  Asynchronous on `stream`.
 */
bsp_status bsp_modal_compute(bsp_plan* plan, const void* delta_k, void* ws, void* stream, double* S);

/*
 * Host helpers of the modal estimator (FP64, no GPU).
 * bsp_modal_radial_powerlaw: table [n_modes][3 (n/2)^2 + 1] of
 *   q_p(k) / sqrt(k P(k)) (sqrt_k != 0, Sec. 3.5) or q_p(k) / sqrt(P(k)),
 *   k = k_f |n|, P(k) = amp k^n_s, q_p the shifted Legendre polynomial P_p on
 *   [kmin, kmax] (zero outside); 0 at n = 0.
 * bsp_modal_modes: the first n_keep 3-D modes (p <= q <= r), ordered by
 *   (p+q+r, p, q, r), as int32 [n_keep][3].
 * bsp_modal_gamma: gamma_nm = <<Q_n | Q_m>> = (1/8 pi^4) int_V dk1 dk2 dk3
 *   Q_n Q_m over the tetrapyd V = {k_i in [kmin, kmax], 2 max k_i <= sum k_i}
 *   (Sec. 3.5), Q_n the symmetrised product of Eq. Qn; piecewise
 *   Gauss-Legendre with npts nodes per piece (exact for polynomial degree
 *   < 2 npts per variable).  gamma is FP64 [n_keep][n_keep].
 * bsp_modal_project: beta = gamma^-1 S for n_rhs right-hand sides
 *   (S, beta: [n_rhs][n_keep]) by Cholesky (Eq. betaCalc); BSP_EINVAL if
 *   gamma is not positive definite.
 */
bsp_status bsp_modal_radial_powerlaw(int n, double box, int n_modes, double kmin, double kmax, double amp,
                                     double n_s, int sqrt_k, double* table);
bsp_status bsp_modal_modes(int n_modes_1d, int n_keep, int32_t* modes);
bsp_status bsp_modal_gamma(int n_keep, const int32_t* modes, double kmin, double kmax, int npts,
                           double* gamma);
bsp_status bsp_modal_project(int n_keep, const double* gamma, int n_rhs, const double* S, double* beta);

/*
 * Batches of mock realisations on uneven grids, and their covariance (the
 * covariance from mock catalogues of Sec. 1 and Sec. 3.1).
 *
 * bsp_batch_create: one plan per grid size (sizes[0..n_sizes), <= 8), same
 *   shells, multipoles and precision (flags 0).
 * bsp_batch_workspace_size: device workspace for prepare and run (one plan
 *   workspace shared by all sizes, two input buffers, a B staging area).
 * bsp_batch_prepare: counts for every size (BSP_EINVAL if the sizes disagree
 *   on the valid bins: rows would not line up); with autotune != 0 times,
 *   per size, the FFT batch {4, 16, 64} against the CUDA-core contraction
 *   grid {1024, 2048, 4096} (BSP_FP32) or the tensor-core tile height
 *   {96, 64} at the default 64-point accumulation chunk (bsp_plan_tune_tc;
 *   longer chunks are less accurate) and keeps the fastest; then
 *   captures bsp_compute into one CUDA graph per (size, input buffer).
 *   Synchronises `stream`.
 * bsp_batch_info / bsp_batch_tuning / bsp_batch_bins: n_bins, the
 *   autotuner's choices and times (arrays of n_sizes; 0 = not tuned), and
 *   the common bins / counts.
 * bsp_batch_run: for m < n_mocks, copies the complex64 half spectrum at host
 *   pointer delta_host[m] (pinned memory for overlap) of grid
 *   sizes[size_index[m]] into an input buffer on an internal copy stream while
 *   the previous mock's graph runs, replays that size's graph on `stream`,
 *   and stores B into rows (device FP64 [n_mocks][n_ell * n_bins]).
 *   Asynchronous on `stream`; the host arrays must stay valid until it
 *   completes.
 * bsp_covariance: mean (device FP64 [d]) and unbiased covariance (device
 *   FP64 [d][d]) of the m >= 2 rows of a device FP64 [m][d] matrix, two
 *   passes (mean, then centred products) in a fixed order.
 */
typedef struct bsp_batch bsp_batch;
bsp_status bsp_batch_create(bsp_batch** out, int n_sizes, const int* sizes, double box, int n_shells,
                            const double* edges_kf, int n_ell, const int* ells, int prec, unsigned flags);
void bsp_batch_destroy(bsp_batch* batch);
bsp_status bsp_batch_workspace_size(const bsp_batch* batch, size_t* bytes);
bsp_status bsp_batch_prepare(bsp_batch* batch, void* ws, void* stream, int autotune);
bsp_status bsp_batch_info(const bsp_batch* batch, int* n_bins, int* tuned_ctas, int* tuned_fb,
                          double* tuned_ms);
bsp_status bsp_batch_tuning(const bsp_batch* batch, int* max_rows, int* chunk_points);
bsp_status bsp_batch_bins(const bsp_batch* batch, int32_t* abc, double* counts);
bsp_status bsp_batch_run(bsp_batch* batch, int n_mocks, const int* size_index, const void* const* delta_host,
                         void* ws, void* stream, double* rows);
bsp_status bsp_covariance(int m, int d, const double* rows, double* mean, double* cov, void* stream);

/* Release the plan and its device tables (NULL is ignored). */
void bsp_plan_destroy(bsp_plan* plan);

/* Bytes of device workspace bsp_counts / bsp_compute need (the maximum of
 * both).  The workspace holds the filtered fields, FFT intermediates and
 * per-block partial sums; its contents need not persist between calls. */
bsp_status bsp_workspace_size(const bsp_plan* plan, size_t* bytes);

/*
 * Triangle counts N_abc (V_B of Sec. 3.1, "similarly evaluated" through unit
 * fields I_a(x) = sum_{n in a} e^{ik.x}, N_abc = n^-3 sum_x I_a I_b I_c),
 * computed in FP64 on the GPU and rounded to integers; geometry only, so
 * one call per plan.  Decides the valid bins (N_abc >= 1) and caches the
 * counts and the contraction schedule in the plan.  Synchronises `stream`.
 *   ws   device workspace of bsp_workspace_size bytes.
 */
bsp_status bsp_counts(bsp_plan* plan, void* ws, void* stream);

/*
 * Copy the counts and valid bins of `src` (after its bsp_counts) into `dst`,
 * a plan of the same grid and shells (any multipoles, precision or
 * BSP_FULL_TENSOR setting), instead of counting again.  Host-side plus small uploads; BSP_EINVAL if the
 * geometries differ, BSP_ESTATE if src has no counts.
 */
bsp_status bsp_plan_share_counts(bsp_plan* dst, const bsp_plan* src);

/*
 * The output bins after bsp_counts: *n_bins always; if abc != NULL the
 * bins as int32 [n_bins][3] (a, b, c), lexicographic (a >= b >= c, or with
 * BSP_FULL_TENSOR every (a; b >= c) described at bsp_plan_create); if
 * counts != NULL the FP64 counts [n_bins].  BSP_ESTATE before bsp_counts.
 */
bsp_status bsp_plan_bins(const bsp_plan* plan, int* n_bins, int32_t* abc, double* counts);

/*
 * Aliasing flag per bin (host only, no GPU).  The FFT contraction computes
 * the periodic sum over q1 + q2 + q3 = 0 (mod n); the paper's closure is
 * q1 + q2 + q3 = 0 (Sec. 3.1, Eq. Bisp_ell_restrict).  The two differ only
 * for bins that can hold wrapped triangles, a nonzero multiple of n; every
 * component of a mode of shell s is below hi_s = edges_kf[s+1] in size, so
 * that needs hi_a + hi_b + hi_c > n.  flags[i] = 1 for such bins (they may
 * hold wrapped triangles), 0 for bins whose sum is exactly the continuum
 * closure's.
 *   n, n_shells, edges_kf  the plan's grid and shells (as bsp_plan_create).
 *   abc      host int32 [n_bins][3] shell indices in [0, n_shells).
 *   flags    host int32 [n_bins] (out).
 * BSP_EINVAL for bad edges or indices.
 */
bsp_status bsp_bins_aliased(int n, int n_shells, const double* edges_kf, int n_bins, const int32_t* abc,
                            int32_t* flags);

/*
 * B^l for every valid bin (Eq. Standard_ell_Estim): enqueue filter ->
 * inverse FFTs -> contraction -> FP64 reduction and normalisation.
 *   delta_k  device, complex64 [n][n][n/2+1] (read only).
 *   nbar     mean number density n_p / V of the particles behind delta for
 *            Poisson shot-noise subtraction, or 0 for none.  The term
 *            subtracted per triangle is (the paper is silent; this is the
 *            Poisson expectation with P_tot = |delta|^2 / V)
 *              w_l(mu_1) [(|d1|^2 + |d2|^2 + |d3|^2)/(V nbar) - 2/nbar^2],
 *            evaluated as three more contractions of the same shape.
 *            Needs a plan created with BSP_SHOT_NOISE (else BSP_EINVAL;
 *            BSP_EUNSUPPORTED on tensor-core plans).
 *   ws       device workspace of bsp_workspace_size bytes.
 *   B        device FP64 [n_ell][n_bins], written.
 * Asynchronous on `stream`; BSP_ESTATE before bsp_counts.
 */
bsp_status bsp_compute(bsp_plan* plan, const void* delta_k, double nbar, void* ws,
                       void* stream, double* B);

/*
 * Same as bsp_compute with host buffers: copies delta_k (host, complex64
 * [n][n][n/2+1]) to a device staging area inside ws, computes, and copies
 * B back to host FP64 [n_ell][n_bins].  Synchronises `stream`.
 * The workspace must be bsp_workspace_size + bsp_host_staging_size bytes.
 */
bsp_status bsp_compute_host(bsp_plan* plan, const void* delta_k_host, double nbar, void* ws,
                            void* stream, double* B_host);
bsp_status bsp_host_staging_size(const bsp_plan* plan, size_t* bytes);

/*
 * Power-spectrum multipoles on the plan's shells (Sec. 2, Eq.
 * PowSpecMultipole, plane-parallel with z the line of sight):
 *   P^l_a = 1/(V N_a) sum_{n in shell a} w_l(mu_n) |delta(n)|^2,
 * N_a the number of modes of the full grid in the shell (the half spectrum
 * counts twice for 0 < n_z < n/2; on the n_z = 0, n/2 planes the Hermitian
 * part is used), w_l = (2l+1) L_l, for the plan's multipoles.  With
 * nbar > 0 the Poisson expectation (1/nbar) (1/N_a) sum w_l(mu_n) is
 * subtracted (the paper does not discuss shot noise).
 *   delta_k: device complex64 [n][n][n/2+1], continuum normalised.
 *   ws:      the plan's workspace (bsp_workspace_size bytes, 256-byte
 *            aligned); its first bytes are overwritten.
 *   P:       device FP64 [n_ell][n_shells] (out).
 *   Nk:      device FP64 [n_shells] mode counts (out), or NULL.
 * Asynchronous on `stream`; deterministic.  Standard plans only (EINVAL for
 * modal plans, NULL pointers or nbar < 0).
 */
bsp_status bsp_power_compute(bsp_plan* plan, const void* delta_k, double nbar, void* ws, void* stream, double* P,
                             double* Nk);

/*
 * The density input the estimators take, from particles: cloud-in-cell
 * assignment on two n^3 grids (cells at j H and at (j + 1/2) H, H = box/n),
 * delta_g = count / (N_p / n^3) - 1, a forward real-to-complex FFT of each,
 * the interlaced average delta(k) = (V/n^3)[X1 + e^{-ik.(H/2)(1,1,1)} X2]/2
 * and the CIC window divided out, prod_a sinc^2(pi n_a / n).  The paper
 * starts from a density grid; this is the standard preparation of one from
 * a particle catalogue (no counterpart in the paper).
 *   pos:      device float32 [n_particles][3], positions in [0, box).
 *   ws:       device workspace of bsp_density_workspace_size(n) bytes,
 *             256-byte aligned (~16 n^3 bytes); ws_bytes its size.
 *   delta_k:  device complex64 [n][n][n/2+1] (out), continuum normalised.
 *   nbar:     host, N_p / V (out), or NULL.
 * n even, of the form 2^a 3^b 5^c (EINVAL otherwise); asynchronous on
 * `stream`.  The deposit uses floating-point atomics, so results vary in the
 * last bits from call to call.
 */
bsp_status bsp_density_workspace_size(int n, size_t* bytes);
bsp_status bsp_density_cic(int n, double box, long long n_particles, const float* pos, void* ws, size_t ws_bytes,
                           void* stream, void* delta_k, double* nbar);

/*
 * Skew-spectrum multipoles on the plan's shells (Sec. 3.3, the estimator
 * under Eq. skewspecQ with Q the convolution):
 *   S^l_a = 1/(V N_a) sum_{n in a} w_l(mu_n) Re[conj Q(n) delta(n)],
 *   Q = transform of delta(x)^2, delta(x) from every mode but the mean,
 * i.e. the shell average of [delta * delta](-k) delta^(l)(k), normalised by
 * 1/V like P^(l) so that its mean is int d^3q/(2 pi)^3 B^(l)(k, q, |k+q|).
 *   delta_k: device complex64 [n][n][n/2+1].
 *   ws:      device workspace of bsp_skew_workspace_size bytes (~20 n^3),
 *            256-byte aligned, separate from the plan's; ws_bytes its size.
 *   S:       device FP64 [n_ell][n_shells] (out); Nk as for bsp_power_compute.
 * Asynchronous on `stream`; deterministic.  Standard plans only; n even with
 * n and n/2 of the form 2^a 3^b 5^c.
 */
bsp_status bsp_skew_workspace_size(const bsp_plan* plan, size_t* bytes);
bsp_status bsp_skew_compute(bsp_plan* plan, const void* delta_k, void* ws, size_t ws_bytes, void* stream, double* S,
                            double* Nk);

/*
 * Integrated-bispectrum multipoles on the plan's shells (Sec. 3.4, the
 * estimator after Eq. iB_expectation, with P^(l) for the multipoles):
 *   iB^l_a = (1/N_s) sum_{i=1}^{N_s} P^l_a,i dbar_i,
 * the box cut into N_s = m^3 cubes of side n/m cells (cube i = (i_x m + i_y) m
 * + i_z, offset (i_x, i_y, i_z) n/m cells), delta(x) the field of every mode
 * of delta_k but the mean, dbar_i its mean over cube i, and P^l_a,i the
 * power-spectrum multipoles of the cube's field taken as periodic (its own
 * transform, V_s = V/m^3, no window correction) on the plan's shells, whose
 * edges stay in units of the whole box's k_f (a cube mode n_s sits at
 * |n| = m |n_s|; shells holding no such mode give iB = 0 and Nk = 0).
 *   delta_k: device complex64 [n][n][n/2+1].
 *   m:       cubes per side, 1 <= m, n % m == 0, side s = n/m even, >= 8 and
 *            of the form 2^a 3^b 5^c (s/2 too), m^3 <= 65535 (EINVAL /
 *            EUNSUPPORTED otherwise).
 *   ws:      device workspace of bsp_ib_workspace_size bytes (~12 n^3),
 *            256-byte aligned, separate from the plan's; ws_bytes its size
 *            (ENOMEM if smaller).
 *   iB:      device FP64 [n_ell][n_shells] (out); Nk: device FP64 [n_shells]
 *            modes per cube in each shell (out), or NULL.
 * Asynchronous on `stream`; deterministic.  Standard plans only.  The first
 * call with a given m uploads the sub-grid's shell table (a synchronous
 * allocation; not inside a graph capture).
 */
bsp_status bsp_ib_workspace_size(const bsp_plan* plan, int m, size_t* bytes);
bsp_status bsp_ib_compute(bsp_plan* plan, const void* delta_k, int m, void* ws, size_t ws_bytes, void* stream,
                          double* iB, double* Nk);

/* Raw sums T^l = sum_x F^l_a F_b F_c of the last bsp_compute (FP64
 * [n_ell][n_bins], device), copied into T (device).  For tests. */
bsp_status bsp_last_raw(const bsp_plan* plan, void* ws, void* stream, double* T);

/*
 * Schedule statistics after bsp_counts, for roofline accounting:
 * st[0] multiply-adds issued per x-point by the contraction (all tiles,
 * all split products), st[1] useful multiply-adds per x-point (n_ell x
 * n_bins), st[2] work items (tiles), st[3] x-segments per work item.
 */
bsp_status bsp_plan_stats(const bsp_plan* plan, double* st);

/*
 * Schedule knobs (the batch runner's autotuner sets them): the number of
 * CTAs the CUDA-core contraction aims at (0 = keep; <= 4096) and the number
 * of fields transformed per FFT launch (0 = keep; capped by the workspace).
 */
bsp_status bsp_plan_tune(bsp_plan* plan, int target_ctas, int fft_batch);

/*
 * Tensor-core schedule knobs (the batch runner's autotuner sets them):
 * max_rows caps the MMA N of a work item (field rows per tile: 32 .. 96, a
 * multiple of 8; 0 = keep; default 96): smaller works mean more, cheaper
 * work items over the same pairs; chunk_points as for
 * bsp_set_accumulation_chunk (0 = keep).  BSP_EUNSUPPORTED on a CUDA-core
 * plan when a knob is set.  Standard plans rebuild their schedule at once
 * when counts exist.
 */
bsp_status bsp_plan_tune_tc(bsp_plan* plan, int max_rows, int chunk_points);

/*
 * Tensor-core paths only: the number of x-points (a multiple of 64, 64 ..
 * 2^20; default 64) summed in an FP32 tensor-memory accumulator before it
 * is added to the FP32 running sum (itself added to FP64 every 8192 points).
 * Every MMA truncates each of its addends to 25 bits below the largest one,
 * so a longer chunk (a larger accumulator) loses more of every product;
 * shorter chunks are more accurate until the running sum's own rounding
 * dominates, and cost more epilogue work.
 */
bsp_status bsp_set_accumulation_chunk(bsp_plan* plan, int points);

/*
 * Tensor-core paths only: the limit, in SM clock cycles, of every wait
 * inside the contraction's pipeline (copies landed, products written, MMAs
 * done, accumulator drained); 0 restores the default
 * (2^33 cycles, about 4 s).  A wait that runs out makes the kernel record
 * the error in the plan's error word (bsp_device_status), stop issuing work,
 * wait for its own copies and MMAs in flight (always with the default limit)
 * and release its tensor memory; the call's outputs are then undefined.
 * For failure-path testing: a limit of a few hundred cycles makes the first
 * wait for a copy run out.  1 <= cycles <= 2^40, or 0.
 */
bsp_status bsp_set_wait_limit(bsp_plan* plan, long long cycles);

/*
 * Error word of the plan's kernels: 0 if no kernel has reported a problem,
 * else a bit mask of bounded waits that gave up (the kernel then stopped
 * early, released its tensor memory and left its outputs undefined).
 * Synchronous (waits for the device).  Returns BSP_ETIMEOUT if nonzero.
 */
bsp_status bsp_device_status(bsp_plan* plan, int* code);

/*
 * Per-phase device timing of bsp_compute with CUDA events recorded on the
 * caller's stream (off by default; the events add no work).
 * bsp_phase_times waits for the last recorded event and returns the summed
 * milliseconds since profiling was switched on or last read:
 * ms[0] filter + inverse FFTs, ms[1] contraction, ms[2] reduction and
 * normalisation; *ncalls profiled calls; *launches kernel launches of one
 * bsp_compute.  Reading resets the sums.
 */
bsp_status bsp_set_profiling(bsp_plan* plan, int on);
bsp_status bsp_phase_times(bsp_plan* plan, double* ms, int* ncalls, int* launches);



/*
 * Triple sums without any device allocation.  The paper has no counterpart:
 * this serves callers that cannot call cudaMalloc -- a host runtime that
 * hands out all device memory from its own fixed pool (an allocation behind
 * its back breaks its accounting, or fails once the pool holds the whole
 * device), or an embedded caller with a hard memory budget that must know,
 * when the library loads, every byte the library will hold.
 *
 *   T[t] = sum_{x < npts} F_i(x) F_j(x) F_k(x),  (i, j, k) = triplets[3t..3t+2],
 *
 * over caller fields F_f = fields + f * npts (device, FP32, [nfields][npts],
 * 16-byte aligned).  triplets is HOST int32 [ntrip][3] with every index in
 * [0, nfields) (checked on the host before anything is enqueued); T is
 * device FP64 [ntrip] (8-byte aligned), written.  Sums use FP32 products
 * folded 64 at a time into compensated FP32 pairs, then FP64 across segments
 * (the same accuracy as the BSP_FP32 contraction).
 *
 * Scratch: a 131 072-triplet list (1.5 MiB) and 2 097 152 FP64 partial sums
 * (16 MiB) live in fixed device arrays that every GPU loading the library
 * holds until the process exits.  ntrip above 131 072 is rejected with
 * BSP_EINVAL.  Every call reuses the same arrays and they keep the last
 * call's contents; nothing in them needs to start at zero (each partial is
 * written before it is read), but calls that overlap on the GPU (different
 * streams, or host threads) race on them.  The first call on each device
 * looks up the arrays' device addresses with cudaGetSymbolAddress, which
 * synchronises with the device.
 *
 * The triplet list is copied with cudaMemcpyAsync on `stream`.  From
 * pageable host memory the call returns once the copy has been staged; from
 * pinned (page-locked) host memory the copy runs when the stream reaches it,
 * so a pinned `triplets` buffer must stay allocated and unchanged until
 * then.  The kernels run asynchronously on `stream`.  CUDA failures return
 * BSP_ECUDA with the CUDA error text in bsp_last_error().
 */
bsp_status bsp_triple_sums_static(const float* fields, size_t npts, int nfields,
                                  const int32_t* triplets, int ntrip, double* T, void* stream);

/*
 * Measured FP32 CUDA-core throughput of the current GPU (no counterpart in
 * the paper; the peak the BSP_FP32 contraction's roofline is quoted
 * against).  One block of 1024 threads per SM, 8 independent FMA chains per
 * thread, `iters` FMAs per chain (a multiple of 16, >= 16); a short warm-up
 * launch, then one launch timed with CUDA events on `stream`.
 *   scratch  device float [n_SM * 1024], overwritten (4-byte aligned).
 *   tflops   host, 2 * FMAs / time in TFLOP/s (out); ms host, the timed
 *            launch's milliseconds (out, may be NULL).
 * Synchronises `stream`.
 */
bsp_status bsp_fp32_fma_peak(int iters, void* stream, float* scratch, double* tflops, double* ms);

/* Human-readable text for a status, and the last CUDA error text seen by
 * this thread ("" if none). */
const char* bsp_status_string(int status);
const char* bsp_last_error(void);

/* Library version: major*10000 + minor*100 + patch. */
int bsp_version(void);

#ifdef __cplusplus
}
#endif
#endif /* BSP_H */
