// How one tcgen05.mma kind::f16 adds 16 products to an FP32 accumulator
// (M = 128, N = 16, K = 16, A from tensor memory, B from shared memory, D
// preset).  The split-product contraction's error model rests on it.  Each A
// row (lane) is one experiment; B[n][k] = 2^-12 for every n, k, so product k
// of row m is a[m][k] * 2^-12 and all 16 columns of D agree.  Prints, per
// lane, the exact sum and the result in ulps of the preset accumulator;
// tests/test_gpu_mma_accumulation.py compiles it, runs it and checks the
// results against the truncation model stated there.
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__global__ void probe(const float* __restrict__ a_vals, const float* __restrict__ d_init, float* __restrict__ out,
                      int* __restrict__ status) {
    __shared__ __align__(1024) uint8_t bsm[2048];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int i = tid; i < 1024; i += 128) reinterpret_cast<__half*>(bsm)[i] = __float2half(0.f);
    __syncthreads();
    // B: N = 16 rows (two 8-row atoms of 1024 B), 128-byte rows, 16-byte chunk j of row r at chunk j ^ r
    for (int e = tid; e < 16 * 16; e += 128) {
        const int n = e / 16, k = e % 16;
        const int atom = n / 8, r = n % 8, chunk = k / 8, within = k % 8;
        const int off = atom * 1024 + r * 128 + ((chunk ^ r) << 4) + within * 2;
        *reinterpret_cast<__half*>(bsm + off) = __float2half(ldexpf(1.f, -12));
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar)), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(64)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const int m = 32 * warp + lane;
    // A: columns [0, 8), column c holds k = 2c (low half) and 2c + 1 (high half)
    uint32_t av[8];
    for (int c = 0; c < 8; ++c) {
        const __half2 h = __floats2half2_rn(a_vals[m * 16 + 2 * c], a_vals[m * 16 + 2 * c + 1]);
        av[c] = *reinterpret_cast<const uint32_t*>(&h);
    }
    uint32_t dv[16];
    for (int j = 0; j < 16; ++j) dv[j] = __float_as_uint(d_init[m]);
    const uint32_t lanebase = tmem + ((uint32_t)(32 * warp) << 16);
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(lanebase),
                 "r"(av[0]), "r"(av[1]), "r"(av[2]), "r"(av[3]), "r"(av[4]), "r"(av[5]), "r"(av[6]), "r"(av[7])
                 : "memory");
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16};" ::"r"(lanebase + 32),
        "r"(dv[0]), "r"(dv[1]), "r"(dv[2]), "r"(dv[3]), "r"(dv[4]), "r"(dv[5]), "r"(dv[6]), "r"(dv[7]), "r"(dv[8]),
        "r"(dv[9]), "r"(dv[10]), "r"(dv[11]), "r"(dv[12]), "r"(dv[13]), "r"(dv[14]), "r"(dv[15])
        : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
        // instruction descriptor: F32 accumulator, A and B FP16, both K-major, N = 16, M = 128
        const uint32_t idesc = (1u << 4) | (0u << 7) | (0u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);
        uint64_t d = 0;
        const uint32_t sa = smem_u32(bsm);
        d |= (uint64_t)((sa >> 4) & 0x3FFFu);
        d |= (uint64_t)1 << 16;
        d |= (uint64_t)((1024u >> 4) & 0x3FFFu) << 32;
        d |= (uint64_t)1 << 46;
        d |= (uint64_t)2 << 61;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(tmem + 32),
            "r"(tmem), "l"(d), "r"(idesc), "r"(1)
            : "memory");
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&bar))
                     : "memory");
    }
    // bounded wait for the MMA (about 1 s)
    bool ok = false;
    const long long t0 = clock64();
    while (!ok) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_u32(&bar)), "r"(0)
            : "memory");
        ok = done != 0;
        if (!ok && clock64() - t0 > (1ll << 31)) break;
    }
    if (!ok && tid == 0) atomicOr(status, 1);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        uint32_t r[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
            "%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(lanebase + 32));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        for (int j = 0; j < 16; ++j) out[m * 16 + j] = __uint_as_float(r[j]);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(64) : "memory");
    }
}

int main() {
    float a[128 * 16] = {0}, d[128] = {0};
    const float q = ldexpf(1.f, -12);
    auto row = [&](int m, float dd, std::initializer_list<float> vals, int reps = 0, float rv = 0.f) {
        d[m] = dd;
        int k = 0;
        for (float v : vals) a[m * 16 + k++] = v;
        for (int i = 0; i < reps; ++i) a[m * 16 + k++] = rv;
    };
    row(0, 1.f, {1.5f * q});
    row(1, 1.f, {}, 16, 0.75f * q);
    row(2, 1.f, {}, 16, -0.75f * q);
    row(3, -1.f, {}, 16, 0.75f * q);
    row(4, 0.f, {4096.f, 1.5f * q});
    row(5, 1.f, {1.5f * 2 * q});
    row(6, 1.f, {}, 16, 0.5f * q);
    row(7, 1.f, {}, 16, 0.25f * q);
    row(8, 1.f, {}, 16, 0.125f * q);
    row(9, 1.f, {-1.25f * q});
    row(10, 1.f, {}, 16, q);
    row(11, 0.f, {4096.f}, 15, 0.75f * q);
    row(12, 0.f, {4096.f}, 15, -0.75f * q);
    row(13, 1.f, {}, 8, 0.75f * q);
    for (int k = 8; k < 16; ++k) a[13 * 16 + k] = -0.75f * q;
    row(14, 1.f, {0.75f * q});
    row(15, 1.f, {}, 3, 0.75f * q);
    row(16, 0.f, {4096.f}, 15, 0.5f * q);
    row(17, ldexpf(1.f, 20), {}, 16, 192.f);          // lane 1 scaled by 2^20
    row(18, 1.f, {}, 16, 0.375f * q);                  // 0.1875 ulp each, sum 3 ulp
    row(19, 1.f, {1.25f * q});                         // 0.625 ulp alone
    row(20, 1.f, {1.75f * q});                         // 0.875 ulp alone
    row(21, 1.f, {0.5f * q, 0.5f * q});                // two half-ulp products
    row(22, 1.f, {}, 4, 0.75f * q);                    // 1.5 ulp from four 0.375 ulp products
    row(23, 1.f, {-0.5f * q});                         // -0.5 * 2^-24: 1 - half an ulp of the binade below
    float *da, *dd, *dout;
    int* dst;
    cudaMalloc(&da, sizeof(a));
    cudaMalloc(&dd, sizeof(d));
    cudaMalloc(&dout, 128 * 16 * sizeof(float));
    cudaMalloc(&dst, sizeof(int));
    cudaMemcpy(da, a, sizeof(a), cudaMemcpyHostToDevice);
    cudaMemcpy(dd, d, sizeof(d), cudaMemcpyHostToDevice);
    cudaMemset(dout, 0, 128 * 16 * sizeof(float));
    cudaMemset(dst, 0, sizeof(int));
    probe<<<1, 128>>>(da, dd, dout, dst);
    cudaError_t e = cudaDeviceSynchronize();
    float out[128 * 16];
    int st = 0;
    cudaMemcpy(out, dout, sizeof(out), cudaMemcpyDeviceToHost);
    cudaMemcpy(&st, dst, sizeof(int), cudaMemcpyDeviceToHost);
    printf("cuda %s status %d\n", cudaGetErrorString(e), st);
    for (int m = 0; m < 24; ++m) {
        double exact = d[m];
        for (int k = 0; k < 16; ++k) exact += (double)__half2float(__float2half(a[m * 16 + k])) * (double)q;
        const float r = out[m * 16];
        bool same = true;
        for (int j = 1; j < 16; ++j) same &= out[m * 16 + j] == r;
        const double u = d[m] != 0.f ? ldexp(1.0, (int)floor(log2(fabs((double)d[m]))) - 23) : ldexp(1.0, -23);
        uint32_t bits;
        memcpy(&bits, &r, 4);
        printf("lane %2d d=%-10g exact-d = %+8.4f ulp(d)   got-d = %+8.4f ulp(d)  (0x%08x)%s\n", m, d[m],
               (exact - d[m]) / u, ((double)r - d[m]) / u, bits, same ? "" : "  COLUMNS DIFFER");
    }
    return e == cudaSuccess && st == 0 ? 0 : 1;
}
