// bsp_tc.cu -- tensor-core (tcgen05) contraction of the filtered fields.
//
// The x-integral of Eq. Standard_ell_Estim (Sec. 3.1),
//   T^l[a; b, c] = sum_x F^l_a(x) F^0_b(x) F^0_c(x),
// is a dense contraction over x once the pair products P_bc = F^0_b F^0_c
// are formed: D[pair][row] = sum_x P_pair(x) F_row(x), rows = fields (l, a).
// A CTA owns one tile -- 128 pairs (the MMA M) times N <= 96 field rows --
// and one x-segment, and runs a warp-specialised pipeline per K-block of 64
// points:
//   warp 0      bulk copies (TMA engine, no tensor map): the F^0 rows (FP32)
//               of the tile's shells and the hi/lo planes of its field
//               groups, stored by the FFT as the swizzled shared-memory image
//               (one copy per contiguous run), four stages deep;
//   warps 4-11  form P = F_b F_c in FP32 (one pair per TMEM lane, half a
//               K-block per warp), split it into 16-bit hi + lo and store
//               both in tensor memory, where the MMA reads its A operand;
//   warp 1      walks the K-blocks (warp-uniform loop state); one elected
//               lane issues tcgen05.mma kind::f16, M=128, K=16, A from
//               tensor memory, B (field planes) from shared memory:
//               D += P_hi F_hi and, in a separate accumulator, E += P_hi F_lo
//               + P_lo F_hi (split products; D alone for the plain 16-bit
//               mode), FP32 accumulators in tensor memory;
//   warps 12-19 drain D every `chunk` K-blocks and E every CORR_KB K-blocks
//               (tcgen05.ld), add them to a running FP32 sum in registers,
//               and every FLUSH_KB K-blocks add that sum, unscaled,
//               to the CTA's FP64 slot in global memory (fire-and-forget
//               reductions).
// Two accumulator buffers and two A buffers in tensor memory keep TMA, the
// CUDA-core prologue, the MMAs and the epilogue overlapped.  Every mbarrier
// wait is bounded; on timeout the CTA records an error code, stops, waits
// (bounded) for its own copies in flight and releases its tensor memory.

#include "bsp_internal.h"

namespace bsp {

namespace {

constexpr int TC_M = 128;        // pairs per tile = MMA M
constexpr int TC_NMAX = 96;      // field rows per tile = MMA N (max)
constexpr int TC_SLOT = 128 * 128;   // FP64 values per CTA slot of the partial sums, [column][pair]
constexpr int TC_KB = 64;        // x-points per K-block (128 bytes of 16-bit values)
constexpr int NT = 4;            // TMA ring stages (F0 rows + field planes)
constexpr int TC_MAXSH = 64;     // F0 rows per tile
#ifndef TC_PRO_WARPS
#define TC_PRO_WARPS 8
#endif
// warps: 0 copies, 1 MMA, 4 .. 4 + N_PRO - 1 pair products (N_PRO / 4 per TMEM
// lane quadrant, each a 64 / (N_PRO / 4)-point part of every K-block), then 8 drain warps
constexpr int N_PRO = TC_PRO_WARPS, PRO_PTS = 64 / (N_PRO / 4), PRO_CH = PRO_PTS / 4;
// 8 drain warps: warp 12 + 4 h + q reads columns [48 h, 48 h + 48) of lane
// quadrant q and keeps their running sum in registers
constexpr int W_TMA = 0, W_MMA = 1, W_PRO0 = 4, W_EPI0 = W_PRO0 + N_PRO, N_EPI = 8, EPI_COLS = 48;
constexpr int TC_THREADS = 32 * (W_EPI0 + N_EPI);
static_assert(N_PRO == 8 || N_PRO == 16, "pair-product warps: 8 or 16");
// tensor memory columns: the P_hi F_hi accumulators D0 [0,96) and D1 [96,192),
// drained every chunk; the correction accumulator E = P_hi F_lo + P_lo F_hi
// [192,288), drained every CORR_KB K-blocks; two A buffers [288,352) and
// [352,416), hi in the first 32 columns, lo in the next 32.  The running FP32
// sum of the drained accumulators lives in the drain warps' registers.
// E's terms are ~2^-11 of D's: kept apart, the tensor core's truncating FP32
// accumulation does not lose half an ulp of D on each correction product.
// With the MMAs issued by an elected lane of the whole warp (below), the 12
// MMAs of a split K-block issue in ~320 cycles and complete ~500 later, so a
// third A buffer no longer shortens the chain products -> MMAs -> products.
constexpr uint32_t TMEM_COLS = 512, COL_ACC = 96, COL_CORR = 192, COL_A = 288;
constexpr int NA = 2;            // A buffers (pair products) in tensor memory
constexpr int CORR_KB = 64;      // K-blocks per drain of E (a multiple of the chunk)
constexpr int FLUSH_KB = 128;    // K-blocks between FP64 flushes of the running sum
constexpr long long WAIT_CYCLES = 1ll << 33;   // ~4 s at 2 GHz

struct TcSmem {
    uint8_t f0[NT][TC_MAXSH * 256];        // [stage][row][64 floats], each half 128-byte swizzled
    uint8_t b[NT][TC_NMAX / 8 * 2048];     // [stage][group of 8 fields][hi 1024 B | lo 1024 B]
    // tma_full: a stage's copies landed; kb_done: the MMAs of K-block k finished
    // (frees TMA stage k % NT and A buffer k % NA); a_full: A buffer written
    // corr_empty: E was read
    uint64_t tma_full[NT], kb_done[NT], a_full[NA], acc_full[2], acc_empty[2], corr_empty;
    uint32_t tmem_base;
    volatile int abort;
    int npc;                  // plane copies per K-block
    int4 pc[16];              // plane copy: (first group in the K-block, first group in the stage, groups, -)
    int2 pf[TC_M];
    float pscale[TC_M];
    float fscale[TC_NMAX];
    int fexp[TC_NMAX];        // -log2 of fscale (the flush scales by 2^(fexp + pexp))
    TcWork w;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
// Has the phase of parity `parity` completed?  test_wait never blocks;
// try_wait may block for a short time set by the hardware.
__device__ __forceinline__ bool mbar_test(uint32_t addr, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    return done != 0;
}
__device__ __forceinline__ bool mbar_try(uint32_t addr, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    return done != 0;
}
// Wait for the phase of parity `parity` to complete; false once `limit` cycles
// have passed (~4 s by default).  After one plain try_wait, waits poll with a
// suspend-time hint: the waiting thread sleeps in the barrier until the phase
// completes (or ~2 us pass) instead of re-reading shared memory in a tight
// loop, which took shared-memory bandwidth from the copies, the pair products
// and the MMAs.  Under a short limit (< 2^20 cycles) the wait polls with
// test_wait instead, so that the limit holds to within a few hundred cycles.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, long long limit = WAIT_CYCLES) {
    const uint32_t addr = smem_u32(b);
    const bool sleep = limit >= (1ll << 20);
    if (sleep ? mbar_try(addr, parity) : mbar_test(addr, parity)) return true;
    const long long t0 = clock64();
    while (true) {
        uint32_t done;
        if (sleep)
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
                " selp.u32 %0, 1, 0, p;\n}\n"
                : "=r"(done)
                : "r"(addr), "r"(parity), "r"(2000u)
                : "memory");
        else
            done = mbar_test(addr, parity);
        if (done) return true;
        if (clock64() - t0 > limit) return false;
    }
}

// 1-D bulk copy global -> shared (16-byte aligned, size a multiple of 16), completing on bar.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D (tensor memory) += A (tensor memory, M x 16, one row per lane) * B (shared memory)^T
__device__ __forceinline__ void mma_ts(uint32_t d, uint32_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
        "r"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_ts2(uint32_t d, uint32_t a, uint32_t blo, uint32_t bhi, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n .reg .b64 bd;\n setp.ne.b32 p, %5, 0;\n mov.b64 bd, {%2, %3};\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], bd, %4, p;\n}\n" ::"r"(d),
        "r"(a), "r"(blo), "r"(bhi), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ bool elect_one() {
    uint32_t e;
    asm volatile("{\n .reg .b32 r;\n .reg .pred p;\n elect.sync r|p, 0xffffffff;\n selp.u32 %0, 1, 0, p;\n}\n" : "=r"(e));
    return e != 0;
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15, %16};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
        "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&r)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
                 "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
                 : "memory");
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand in 8-row x 128-byte atoms
// with the 128-byte swizzle, atoms `sbo` bytes apart (stride byte offset).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);   // start address >> 4
    d |= (uint64_t)1 << 16;                     // leading byte offset (unused with this swizzle)
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;   // stride byte offset >> 4
    d |= (uint64_t)1 << 46;                     // descriptor version (0b001)
    d |= (uint64_t)2 << 61;                     // 128-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator, A and B of the same
// 16-bit type (0 = FP16, 1 = BF16), both K-major, M = 128.
__host__ __device__ constexpr uint32_t make_idesc(uint32_t fmt, uint32_t n) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((n >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
}

// Two FP32 values -> packed 16-bit pair (x0 in the low half), round to nearest even.
template <bool F16>
__device__ __forceinline__ uint32_t pack2(float x0, float x1) {
    uint32_t r;
    if (F16) asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(x1), "f"(x0));
    else asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(x1), "f"(x0));
    return r;
}
template <bool F16>
__device__ __forceinline__ void unpack2(uint32_t v, float& x0, float& x1) {
    if (F16) {
        unsigned short l = (unsigned short)(v & 0xFFFFu), h = (unsigned short)(v >> 16);
        asm("cvt.f32.f16 %0, %1;" : "=f"(x0) : "h"(l));
        asm("cvt.f32.f16 %0, %1;" : "=f"(x1) : "h"(h));
    } else {
        x0 = __uint_as_float(v << 16);
        x1 = __uint_as_float(v & 0xFFFF0000u);
    }
}

// Power of two s with bound * s in [2^(t-1), 2^t) (the FFT's pass 3 applies
// the same scales: t = 15 to the 16-bit planes, t = 7 to the FP32 pair factors).
__device__ __forceinline__ float pow2_scale(float bound, int t = 15) {
    if (!(bound > 0.f)) return 1.f;
    int e;
    frexpf(bound, &e);
    return ldexpf(1.f, t - e);
}

__device__ __forceinline__ uint64_t fmul2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t fsub2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t pack64(float x0, float x1) {
    uint64_t d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(x0), "f"(x1));
    return d;
}
__device__ __forceinline__ void unpack64(uint64_t v, float& x0, float& x1) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(x0), "=f"(x1) : "l"(v));
}

// f * 2^k as a double, built from the float's bits with integer operations
// (k is small: |k| < 300).  The FP64 pipe of this GPU is slow; the flushes
// used to divide by the scale in FP64, which cost more than the MMAs.
// Zero, denormal, infinite and NaN inputs take the exact library path.
__device__ __forceinline__ double f32_ldexp_f64(float f, int k) {
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xFFu;
    if (e == 0u || e == 0xFFu) return ldexp((double)f, k);
    const unsigned long long b = ((unsigned long long)(u >> 31) << 63) |
                                 ((unsigned long long)(e + 896u + (uint32_t)k) << 52) |
                                 ((unsigned long long)(u & 0x7FFFFFu) << 29);
    return __longlong_as_double((long long)b);
}

__device__ __forceinline__ void set_abort(TcSmem& S, int* err, int code) {
    S.abort = 1;
    atomicOr(err, code);
}

template <bool F16>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_contract_tc(const float* __restrict__ gf0, int f0_rows, int f0_row0, const uint32_t* __restrict__ gplanes,
                  int groups, long long nkb_real, const TcWork* __restrict__ works,
                  const int2* __restrict__ pair_shells, int pair_base,
                  const unsigned* __restrict__ fmax2, float bound_mul, const TcUnit* __restrict__ units,
                  int lsup, int nsup, int nprod, int CHUNK, double* __restrict__ partial,
                  int* __restrict__ err, long long wlim) {
    extern __shared__ uint8_t smem_raw[];
    TcSmem& S = *reinterpret_cast<TcSmem*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const TcUnit unit = units[blockIdx.x];
    if (tid < (int)(sizeof(TcWork) / sizeof(int)))
        reinterpret_cast<int*>(&S.w)[tid] = reinterpret_cast<const int*>(works + unit.work)[tid];
    __syncthreads();
    const TcWork& w = S.w;
    // iteration k covers K-block (k / len) * lsup + start + k % len: every CTA
    // walks the super-segments in the same order (shared fields stay in L2);
    // K-blocks past the end of the grid load as zeros and add nothing
    const int nkb = nsup * unit.len;
    const int nch = (nkb + CHUNK - 1) / CHUNK;
    const int FL = max(1, FLUSH_KB / CHUNK);   // chunks per FP64 flush
    const int CC = max(1, CORR_KB / CHUNK);    // chunks per drain of E
    const uint32_t N = (uint32_t)w.n;

    if (tid == 0) {
        for (int s = 0; s < NT; ++s) {
            mbar_init(&S.tma_full[s], 1);
            mbar_init(&S.kb_done[s], 1);
        }
        for (int j = 0; j < NA; ++j) mbar_init(&S.a_full[j], N_PRO);
        for (int j = 0; j < 2; ++j) {
            mbar_init(&S.acc_full[j], 1);
            mbar_init(&S.acc_empty[j], N_EPI);
        }
        mbar_init(&S.corr_empty, N_EPI);
        S.abort = 0;
        // field-plane copies: one per run of consecutive groups
        int npc = 0;
        for (int j = 0; j < w.nbox;) {
            int L = 1;
            while (j + L < w.nbox && w.box_field[j + L] == w.box_field[j] + 8 * L) ++L;
            S.pc[npc++] = make_int4(w.box_field[j] >> 3, j, L, 0);
            j += L;
        }
        S.npc = npc;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // zero every stage once: MMA rows past the tile's groups (N rounds 8 nbox up
    // to 16) and K-blocks past the end of the grid (no copies) then read zeros
    for (int i = tid; i < (int)(sizeof(S.f0) + sizeof(S.b)) / 16; i += TC_THREADS)
        reinterpret_cast<uint4*>(S.f0)[i] = make_uint4(0u, 0u, 0u, 0u);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (tid < TC_M) {
        int2 v = {-1, -1};
        float sc = 1.f;
        if (tid < w.npairs) {
            v = pair_shells[w.pair0 + tid];
            // the FP32 pair factors arrive pre-scaled by s7 each (|F s7| < 2^7): the
            // pair product carries s7_b s7_c, undone at the end
            sc = pow2_scale(bound_mul * __uint_as_float(fmax2[pair_base + v.x]), 7) *
                 pow2_scale(bound_mul * __uint_as_float(fmax2[pair_base + v.y]), 7);
            v.x -= w.shell_lo;
            v.y -= w.shell_lo;
        }
        S.pf[tid] = v;
        S.pscale[tid] = sc;
    } else if (tid < TC_M + TC_NMAX) {
        // the scale the FFT applied to this field row's 16-bit planes
        const int c = tid - TC_M;
        float fs = 1.f;
        if (c < 8 * w.nbox) fs = pow2_scale(bound_mul * __uint_as_float(fmax2[w.box_field[c >> 3] + (c & 7)]));
        S.fscale[c] = fs;
        S.fexp[c] = -ilogbf(fs);
    }
    if (warp == W_MMA) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&S.tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem_base;

    if (warp == W_TMA) {
        if (lane == 0) {
            const int npc = S.npc;
            const uint32_t f0_bytes = (uint32_t)w.nshell * 256;
            const uint32_t bytes = f0_bytes + (uint32_t)w.nbox * 2048;
            const uint8_t* f0src = reinterpret_cast<const uint8_t*>(gf0) + (size_t)(f0_row0 + w.shell_lo) * 256;
            const uint8_t* psrc = reinterpret_cast<const uint8_t*>(gplanes);
            int issued = 0;
            for (int k = 0; k < nkb && !S.abort; ++k) {
                const int s = k % NT, u = k / NT;
                if (u > 0 && !mbar_wait(&S.kb_done[s], (u - 1) & 1, wlim)) {
                    set_abort(S, err, 1);
                    break;
                }
                const int sup = k / unit.len, kin = k % unit.len;
                const long long kb = (long long)sup * lsup + unit.start + kin;
                if (kb < nkb_real) {
                    mbar_expect_tx(&S.tma_full[s], bytes);
                    bulk_load(S.f0[s], f0src + (size_t)kb * f0_rows * 256, f0_bytes, &S.tma_full[s]);
                    for (int j = 0; j < npc; ++j) {
                        const int4 c = S.pc[j];
                        bulk_load(&S.b[s][c.y * 2048], psrc + ((size_t)kb * groups + c.x) * 2048,
                                  (uint32_t)c.z * 2048, &S.tma_full[s]);
                    }
                } else {
                    mbar_expect_tx(&S.tma_full[s], 0);   // past the grid: nothing to load
                }
                issued = k + 1;
            }
            // copies in flight must land before the CTA can exit: the last use of each
            // stage (always the long limit, whatever the pipeline waits use)
            for (int k = max(0, issued - NT); k < issued; ++k)
                if (!mbar_wait(&S.tma_full[k % NT], (k / NT) & 1)) atomicOr(err, 16);
        }
    } else if (warp == W_MMA) {
        // the whole warp walks the K-blocks (the loop state stays warp-uniform);
        // one elected lane issues the MMAs and commits
        const uint32_t idesc = make_idesc(F16 ? 0u : 1u, N);
        // B descriptors: the high word is fixed (stride, version, swizzle), the low
        // word is the start address >> 4: stage s, slice kk, half h at
        // dlo0 + s * (stage bytes >> 4) + 2 kk + 64 h
        const uint32_t dhi = (uint32_t)(sw128_desc(0u, 2048) >> 32);
        const uint32_t dlo0 = (uint32_t)sw128_desc(smem_u32(S.b[0]), 2048);
        constexpr uint32_t STAGE16 = (uint32_t)(sizeof(S.b[0]) >> 4);
        int done = 0, kc = 0, c = 0;   // kc = k % CHUNK, c = k / CHUNK
        bool ok = true;
        for (int k = 0; k < nkb; ++k) {
            const int s = k % NT, u = k / NT, sa = k % NA;
            const int j = c & 1;
            const bool efirst = kc == 0 && c % CC == 0;   // first K-block of a drain period of E
            if (kc == 0 && c >= 2 && !__all_sync(0xffffffffu, mbar_wait(&S.acc_empty[j], ((c >> 1) - 1) & 1, wlim))) {
                ok = false;
                break;
            }
            if (nprod == 3 && efirst && c > 0 &&
                !__all_sync(0xffffffffu, mbar_wait(&S.corr_empty, ((c / CC) - 1) & 1, wlim))) {
                ok = false;
                break;
            }
            if (!__all_sync(0xffffffffu, mbar_wait(&S.tma_full[s], u & 1, wlim) && mbar_wait(&S.a_full[sa], (k / NA) & 1, wlim))) {
                if (lane == 0) set_abort(S, err, 4);
                break;
            }
            if (__shfl_sync(0xffffffffu, S.abort, 0)) break;
            tc_fence_after();
            if (elect_one()) {
                const uint32_t d = tmem + (uint32_t)j * COL_ACC, de = tmem + COL_CORR;
                const uint32_t ah = tmem + COL_A + (uint32_t)sa * 64, al = ah + 32;
                const uint32_t lh = dlo0 + (uint32_t)s * STAGE16;
#pragma unroll
                for (int kk = 0; kk < TC_KB / 16; ++kk) {
                    const uint32_t oa = (uint32_t)kk * 8, ob = (uint32_t)kk * 2;
                    mma_ts2(d, ah + oa, lh + ob, dhi, idesc, (kc == 0 && kk == 0) ? 0u : 1u);
                    if (nprod == 3) {
                        mma_ts2(de, ah + oa, lh + 64u + ob, dhi, idesc, (efirst && kk == 0) ? 0u : 1u);
                        mma_ts2(de, al + oa, lh + ob, dhi, idesc, 1u);
                    }
                }
                mma_commit(&S.kb_done[s]);
                if (kc + 1 == CHUNK || k == nkb - 1) mma_commit(&S.acc_full[j]);
            }
            __syncwarp();
            if (++kc == CHUNK || k == nkb - 1) {
                kc = 0;
                ++c;
            }
            done = k + 1;
        }
        if (!ok && lane == 0) set_abort(S, err, 2);
        // the last MMAs must finish before tensor memory is released (long limit)
        if (done > 0 && !__all_sync(0xffffffffu, mbar_wait(&S.kb_done[(done - 1) % NT], ((done - 1) / NT) & 1)) && lane == 0)
            atomicOr(err, 32);
    } else if (warp >= W_PRO0 && warp < W_PRO0 + N_PRO) {
        // lane quadrant q of tensor memory = pairs 32 q .. 32 q + 31; part t of each
        // K-block: points t * PRO_PTS .., 16-byte chunks j0 .. j0 + PRO_CH - 1 of F0 half h
        const int q = warp & 3, t = (warp - W_PRO0) >> 2, h = (t * PRO_PTS) >> 5, j0 = ((t * PRO_PTS) & 31) >> 2;
        const int i = 32 * q + lane;
        const int2 bc = S.pf[i];
        const bool pair = bc.x >= 0;
        const int rb = pair ? bc.x : 0, rc = pair ? bc.y : 0;
        // F0 row r (relative to the tile's first shell, absolute K-block row g = f0_row0 +
        // shell_lo + r): 16-byte chunk j of half h at r*256 + 128 h + ((j ^ (g & 7)) << 4)
        const int g0 = f0_row0 + w.shell_lo;
        const int ob = rb * 256 + 128 * h, sb = (g0 + rb) & 7, oc = rc * 256 + 128 * h, sc = (g0 + rc) & 7;
        const uint32_t lanebase = ((uint32_t)(32 * q) << 16) + (uint32_t)(t * PRO_PTS / 2);
        for (int k = 0; k < nkb && !S.abort; ++k) {
            const int s = k % NT, u = k / NT, sa = k % NA;
            if (!mbar_wait(&S.tma_full[s], u & 1, wlim) ||
                (k >= NA && !mbar_wait(&S.kb_done[(k - NA) % NT], ((k - NA) / NT) & 1, wlim))) {
                set_abort(S, err, 8);
                break;
            }
            tc_fence_after();
            const bool live = pair && (long long)(k / unit.len) * lsup + unit.start + k % unit.len < nkb_real;
            const uint8_t* f0 = S.f0[s];
            uint32_t vh[2 * PRO_CH], vl[2 * PRO_CH];
#pragma unroll
            for (int jj = 0; jj < PRO_CH; ++jj) {
                const int j = j0 + jj;
                uint64_t p01 = 0, p23 = 0;
                if (live) {
                    const float4 fb = *reinterpret_cast<const float4*>(f0 + ob + ((j ^ sb) << 4));
                    const float4 fc = *reinterpret_cast<const float4*>(f0 + oc + ((j ^ sc) << 4));
                    p01 = fmul2(pack64(fb.x, fb.y), pack64(fc.x, fc.y));
                    p23 = fmul2(pack64(fb.z, fb.w), pack64(fc.z, fc.w));
                }
                float p0, p1, p2, p3, h0, h1, h2, h3;
                unpack64(p01, p0, p1);
                unpack64(p23, p2, p3);
                vh[2 * jj] = pack2<F16>(p0, p1);
                vh[2 * jj + 1] = pack2<F16>(p2, p3);
                unpack2<F16>(vh[2 * jj], h0, h1);
                unpack2<F16>(vh[2 * jj + 1], h2, h3);
                float r0, r1, r2, r3;
                unpack64(fsub2(p01, pack64(h0, h1)), r0, r1);
                unpack64(fsub2(p23, pack64(h2, h3)), r2, r3);
                vl[2 * jj] = pack2<F16>(r0, r1);
                vl[2 * jj + 1] = pack2<F16>(r2, r3);
            }
            const uint32_t ta = tmem + lanebase + COL_A + (uint32_t)sa * 64;
            if constexpr (PRO_CH == 4) {
                tmem_st8(ta, *reinterpret_cast<const uint32_t(*)[8]>(vh));
                if (nprod == 3) tmem_st8(ta + 32, *reinterpret_cast<const uint32_t(*)[8]>(vl));
            } else {
                tmem_st16(ta, *reinterpret_cast<const uint32_t(*)[16]>(vh));
                if (nprod == 3) tmem_st16(ta + 32, *reinterpret_cast<const uint32_t(*)[16]>(vl));
            }
            tmem_st_wait();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&S.a_full[sa]);
        }
    } else if (warp >= W_EPI0) {
        const int q = warp & 3, hc = (warp - W_EPI0) >> 2;
        const uint32_t lanebase = tmem + ((uint32_t)(32 * q) << 16);
        const int row = 32 * q + lane;
        const uint32_t c0 = (uint32_t)(EPI_COLS * hc);   // this warp's columns [c0, c0 + 48) within N
        // the CTA's FP64 slot, [column][pair] (zeroed before the launch): the flushes are
        // fire-and-forget reductions, coalesced over the warp's 32 pairs
        double* dst = partial + (size_t)blockIdx.x * TC_SLOT + row;
        const int pexp = -ilogbf(S.pscale[row]);   // the scales are powers of two
        float sum[EPI_COLS];
#pragma unroll
        for (int t = 0; t < EPI_COLS; ++t) sum[t] = 0.f;
        for (int c = 0; c < nch && !S.abort; ++c) {
            const int j = c & 1, g = c % FL;
            const bool flush = g == FL - 1 || c == nch - 1;
            if (!mbar_wait(&S.acc_full[j], (c >> 1) & 1, wlim)) {
                set_abort(S, err, 64);
                break;
            }
            tc_fence_after();
            // every CC chunks, and at the end, E joins the running sum first
            if (nprod == 3 && ((c + 1) % CC == 0 || c == nch - 1)) {
#pragma unroll
                for (int cg = 0; cg < EPI_COLS / 16; ++cg) {
                    const uint32_t col = c0 + 16u * cg;
                    if (col < N) {
                        uint32_t a[16];
                        tmem_ld16(lanebase + COL_CORR + col, a);
                        tmem_ld_wait();
#pragma unroll
                        for (int t = 0; t < 16; ++t) sum[16 * cg + t] += __uint_as_float(a[t]);
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&S.corr_empty);
            }
            // D joins the running sum; the accumulator is released as soon as it is read
#pragma unroll
            for (int cg = 0; cg < EPI_COLS / 16; ++cg) {
                const uint32_t col = c0 + 16u * cg;
                if (col < N) {
                    uint32_t a[16];
                    tmem_ld16(lanebase + (uint32_t)j * COL_ACC + col, a);
                    tmem_ld_wait();
#pragma unroll
                    for (int t = 0; t < 16; ++t) sum[16 * cg + t] += __uint_as_float(a[t]);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&S.acc_empty[j]);
            if (flush) {
                // the running sum to the CTA's FP64 slot, while the MMAs fill the other D buffer
#pragma unroll
                for (int t = 0; t < EPI_COLS; ++t) {
                    const uint32_t col = c0 + (uint32_t)t;
                    if (col < N) {
                        const double v = f32_ldexp_f64(sum[t], pexp + S.fexp[col]);
                        asm volatile("red.global.add.f64 [%0], %1;" ::"l"(dst + (size_t)col * TC_M), "d"(v)
                                     : "memory");
                    }
                    sum[t] = 0.f;
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == W_MMA) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS)
                     : "memory");
    }
}

}  // namespace

size_t tc_smem_bytes() { return sizeof(TcSmem) + 1024; }

cudaError_t launch_contract_tc(bool f16, const float* f0, int f0_rows, int f0_row0, const uint32_t* planes,
                               int groups, long long nkb, const TcWork* works, const TcUnit* units, int nunits,
                               int lsup, int nsup, const int2* pair_shells, int pair_base, const unsigned* fmax2,
                               float bound_mul, int nprod, int chunk_kb, double* partial, int* err,
                               cudaStream_t st, long long wait_cycles) {
    const size_t smem = tc_smem_bytes();
    const long long wlim = wait_cycles > 0 ? wait_cycles : WAIT_CYCLES;
    static bool set16 = false, setb = false;   // once per kernel, never inside a graph capture
    auto kern = f16 ? k_contract_tc<true> : k_contract_tc<false>;
    cudaError_t e;
    bool& set = f16 ? set16 : setb;
    if (!set) {
        if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return e;
        set = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)nunits);
    cfg.blockDim = dim3(TC_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    return cudaLaunchKernelEx(&cfg, kern, f0, f0_rows, f0_row0, planes, groups, nkb, works, pair_shells, pair_base, fmax2, bound_mul, units, lsup, nsup,
                              nprod, chunk_kb, partial, err, wlim);
}

}  // namespace bsp
