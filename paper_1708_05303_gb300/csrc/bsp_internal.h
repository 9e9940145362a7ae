// bsp_internal.h -- declarations shared by the libbsp translation units.
// Not part of the public ABI (include/bsp.h is).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/bsp.h"

namespace bsp {

// Record `where: <CUDA error text>` as this thread's bsp_last_error() and
// return BSP_ECUDA (defined in bsp_api.cu).
bsp_status record_cuda_error(cudaError_t e, const char* where);

template <typename R>
struct __align__(2 * sizeof(R)) cx {
    R re, im;
};

// What a filtered field is made of (Sec. 3.1 D_k^{(l)}, Sec. 3.5 M^{(l)}_n).
enum FieldKind : int {
    FIELD_DELTA = 0,    // w_l(mu) 1[n in shell] delta(n)
    FIELD_UNIT = 1,     // w_l(mu) 1[n in shell]            (counts: delta == 1)
    FIELD_POWER = 2,    // w_l(mu) 1[n in shell] |delta(n)|^2  (shot noise)
    FIELD_RADIAL = 3,   // w_l(mu) R_p[n^2] delta(n)        (modal)
    FIELD_RAW = 4,      // delta(n) on every mode but the mean (skew spectrum)
};

struct FieldDesc {
    int shell;   // shell index (FIELD_DELTA/UNIT/POWER) or radial table row (FIELD_RADIAL)
    int ell;     // 0, 2, 4
    int kind;    // FieldKind
    int out32;   // index of the FP32/FP64 output field, or -1
    int out16;   // index of the 16-bit hi/lo output planes, or -1
    // the field's spectrum vanishes where any |frequency component| > kext
    // (its shell's outer edge); <= 0: the plan's extent K.  Pass 1 skips the
    // pencils beyond it and passes 2 and 3 read nothing beyond it.
    int kext;
    int pad[2];
};

// Geometry of the pruned inverse FFT.  Only frequencies |f| <= K per axis
// can be nonzero (all filters vanish for |n| >= the last edge).
struct FftGeom {
    int n;        // grid side
    int K;        // largest kept |frequency| on x, y (pruned) -- n/2 when not pruned
    int nK;       // kept x/y frequencies: 2K+1 (pruned) or n
    int pruned;   // 1 if nK < n
    int nKz;      // kept z frequencies 0..nKz-1 (<= n/2+1)
    int n2max;    // largest |n|^2 in the shell table
    int nrad;     // radix stages for length n
    int rad[8];
    int nrad_h;   // radix stages for length n/2 (real-output pass)
    int rad_h[8];
};

// One contraction work item: a tile of pairs (b, c) (contiguous indices in
// the pair table) times a chunk of up to 64 rows (l, a).
struct Work {
    int pair0;    // first pair index
    int npairs;   // <= 128
    int row0;     // first row of the tile's (l, a) row list
    int nrows;    // <= 64
    int rowbase;  // index into the row-field table of row 0 of this chunk
    int shell_lo; // lowest shell used by the pairs
    int nshell;   // shells shell_lo .. shell_lo + nshell - 1 (<= 64)
    int pad;
};

// One tensor-core work item: 128 pairs x N field rows (N = 8 nbox rounded up to 16).
struct TcWork {
    int pair0, npairs;      // pairs [pair0, pair0 + npairs), npairs <= 128
    int shell_lo, nshell;   // F0 rows the pairs use, nshell <= 64
    int nbox;               // boxes of 8 consecutive field rows
    int n;                  // MMA N
    int pad[2];
    int box_field[16];      // first field (plane index, a multiple of 8) of each box
};

// One persistent tensor-core CTA: the x-range is swept in super-segments of
// `lsup` K-blocks in the same order by every CTA; this CTA handles K-blocks
// [start, start + len) of each super-segment for work item `work`.
struct TcUnit {
    int work;
    int start;
    int len;
    int pad;
};

struct BinLoc {   // where T of (l, bin) lives in the partial buffer
    int work;     // work item (or first partial slot, see k_reduce)
    int row;      // row within the work item
    int col;      // pair within the work item
    int pad;      // number of partial slots to sum when the caller passes nsplit <= 0
};

// Output layout of the real fields.  Field-major (rows32 = groups16 = 0):
// field f at out + f * out_stride (FP32/FP64) and at plane f of hi/lo.
// K-block-major (the tensor-core operands; x is cut into K-blocks of 64
// points, each stored as the shared-memory image the contraction copies):
//   FP32: K-block kb of row r (= out32) is the 256-byte row kb * rows32 + r
//         of a [K-blocks * rows32][64] array; 16-byte chunk J of a row sits
//         at chunk (J & 8) | ((J & 7) ^ (r & 7)) (the 128-byte swizzle of
//         each half);
//   16-bit planes: fields come in groups of 8; K-block kb of group g is the
//         2048 bytes at (kb * groups16 + g) * 2048 of `hi`: the 8 hi rows
//         (128 bytes each) then the 8 lo rows, chunk j of row r at chunk
//         j ^ r (the 128-byte swizzle of the tensor-core operand).
struct FieldLayout {
    int rows32 = 0;
    int groups16 = 0;
};

// ---- launchers (bsp_fft.cu) ----
template <typename R>
cudaError_t launch_fft_fields(const FftGeom& g, const cx<float>* delta, const int16_t* shell_of,
                              const float* radial, const FieldDesc* d_fields, int nfields,
                              const cx<R>* tw, cx<R>* t1, cx<R>* t2, R* out, size_t out_stride,
                              uint32_t* hi, uint32_t* lo, int f16, unsigned* fmax2, unsigned* f0max,
                              cudaStream_t st, FieldLayout lay = FieldLayout());

// Shot-noise combination in the reduction: v -= sum_t coef[t] * (sum of partial set t).
struct ShotTerms {
    int n;
    const double* partial[3];
    double coef[3];
};

// ---- launchers (bsp_contract.cu) ----
template <typename R>
cudaError_t launch_contract_cc(const R* rows, const R* px, const R* py, int sym, size_t fstride,
                               const Work* works, int nwork, const int2* pair_fields,
                               const int* row_fields, size_t npts, int nsplit, double* partial,
                               cudaStream_t st);

// Counts on the cubic group's orbit representatives: wrows[a][r] = w[r] *
// fields[a][idx[r]], urows[a][r] = fields[a][idx[r]] (FP64, [nsh][nrep]).
cudaError_t launch_gather_reps(const double* fields, size_t npts, int nsh, const uint32_t* idx, const double* w,
                               size_t nrep, double* wrows, double* urows, cudaStream_t st);

cudaError_t launch_reduce(const double* partial, int nsplit, size_t unit, int row_stride,
                          const BinLoc* loc, int nout, int nbins, const double* counts, double scale,
                          int mode, double* T_out, double* out, cudaStream_t st,
                          const ShotTerms* shot = nullptr);

// ---- launchers (bsp_tc.cu) ----
// Operands in the K-block-major layout (FieldLayout): F0 row of shell s in
// K-block kb is row kb * f0_rows + f0_row0 + s of f0; the 16-bit planes have
// `groups` groups of 8 fields per K-block; works name fields by plane index.
size_t tc_smem_bytes();
cudaError_t launch_contract_tc(bool f16, const float* f0, int f0_rows, int f0_row0, const uint32_t* planes,
                               int groups, long long nkb, const TcWork* works, const TcUnit* units, int nunits,
                               int lsup, int nsup, const int2* pair_shells, int pair_base, const unsigned* fmax2,
                               float bound_mul, int nprod, int chunk_kb, double* partial, int* err,
                               cudaStream_t st, long long wait_cycles = 0);

// ---- density input stage (bsp_fft.cu) ----
struct DensityLayout {   // byte offsets in the caller's workspace
    size_t tw, grids, spec, end;
};
DensityLayout density_layout(int n);
cudaError_t launch_density(const FftGeom& g, const float* pos, long long np, double box, void* ws,
                           cx<float>* out, cudaStream_t st);
// Forward real-to-complex FFT (unnormalised, e^{-ik.x}) of a * x^2 for a real
// field x [n][n][n]; spectrum T [n][n][n/2+1]; tw = exp(+2 pi i t/n), t < n.
cudaError_t launch_forward_square(const FftGeom& g, const float* x, float a, const cx<float>* tw, cx<float>* T,
                                  cudaStream_t st);
// Forward real-to-complex FFTs of the m^3 sub-cubes of side s = n/m of a real
// field x [n][n][n] (g: the geometry of side s), each scaled by a:
// T [m^3][s][s][s/2+1], cube c = (c_x m + c_y) m + c_z at x offset (c_x s,
// c_y s, c_z s); tw (workspace, s entries) receives exp(+2 pi i t/s).
cudaError_t launch_forward_subcubes(const FftGeom& g, int nfull, int m, const float* x, float a, cx<float>* tw,
                                    cx<float>* T, cudaStream_t st);

// ---- launchers (bsp_power.cu) ----
struct PowerEll {   // the multipoles of a power-spectrum call (even l in {0, 2, 4})
    int n;
    int ell[3];
};
size_t power_partial_bytes(int nblocks, int nsh, int nell);
// P^l_a (Q == nullptr: w_l |delta|^2) or the cross spectrum (w_l Re conj(Q) delta,
// Q in the half-spectrum layout of delta, multiplied by num_scale), over V N_a.
// With nbatch > 1, delta holds nbatch spectra bstride elements apart, each
// summed by nblocks CTAs (partial: nbatch * nblocks slots); with dc_weight
// every product of spectrum b is multiplied by Re delta_b(0), and Nk is the
// count per spectrum.  Rows with f_x^2 + f_y^2 > n2top (the largest |n|^2 of
// any shell, or g.n2max) are skipped.
cudaError_t launch_power(const cx<float>* delta, const cx<float>* Q, double num_scale, const FftGeom& g,
                         const int16_t* shell_of, int nsh, const PowerEll& ells, double V, double nbar, int nblocks,
                         double* partial, double* P, double* Nk, cudaStream_t st, int nbatch = 1,
                         size_t bstride = 0, int dc_weight = 0, int n2top = 1 << 30);

// ---- launchers (bsp_modal.cu) ----
cudaError_t launch_modal_assemble(const double* T, const double* U, const int* ells, int n_ell, int nf,
                                  long long nall, int ntrip, double scale, double* S, cudaStream_t st);

}  // namespace bsp
