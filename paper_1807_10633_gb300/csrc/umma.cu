// G = C_v C_occ^-1 on the 5th-generation tensor cores (tcgen05, TF32) with a split-precision
// correction, for the mixed-form refresh of the walker tables (Sec. III.B, Eq. R).
//
// Per (walker, spin) CTA of four warps:
//   A (M = 128 rows >= n_virt, K = n): rows of C (FP32 copy) for the walker's virtual orbitals;
//   B (N = n rounded up to 16, K = n):  rows of C_occ^-1 transposed (AinvT[c][x], K-major);
//   D = A_hi B_hi + A_hi B_lo + A_lo B_hi  (x_hi = x truncated to TF32, x_lo = x - x_hi),
// accumulated in FP32 in tensor memory, which recovers ~22 bits from TF32 products.  Operands
// are staged in shared memory in the no-swizzle K-major core-matrix layout (8 rows x 16 bytes per
// core matrix); one thread issues the MMAs and commits them to an mbarrier whose wait is bounded
// (on timeout the kernel latches VMC_ERR_TIMEOUT, frees its tensor memory and returns).
#include <stdint.h>

#include "common.cuh"

namespace {

constexpr int kM = 128;          // MMA rows (virtual slots, padded)
constexpr int kThreads = 128;    // four warps: one per 32 tensor-memory lanes
constexpr unsigned kMaxSpin = 1u << 20;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start, leading (K) and stride (row-group) byte offsets,
// descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor: D = F32, A = B = TF32, both K-major, N and M.
__device__ __forceinline__ uint32_t make_idesc(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// byte offset of element (row, k) in a K-major no-swizzle tile with kp4 = K/4 core matrices per row group
__device__ __forceinline__ uint32_t core_off(int row, int k, int kp4) {
    return (uint32_t)((row >> 3) * kp4 * 128 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ void split_tf32(float v, float &hi, float &lo) {
    hi = __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
    lo = v - hi;
}

__global__ void __launch_bounds__(kThreads)
k_g_umma(int M, int na, int nb, const float *__restrict__ Cf, const uint16_t *__restrict__ virt_list,
         const float *__restrict__ AinvT, float *__restrict__ G, unsigned *status, int lbo_k_major) {
    const int w = blockIdx.x, sg = blockIdx.y;
    const int n = sg ? nb : na, nv = M - n;
    const int ne = na + nb;
    if (n == 0 || nv == 0) return;
    const int Kp = (n + 7) & ~7, Np = (n + 15) & ~15, kp4 = Kp >> 2;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    extern __shared__ __align__(1024) unsigned char sm[];
    const uint32_t a_bytes = (uint32_t)(kM / 8) * kp4 * 128, b_bytes = (uint32_t)(Np / 8) * kp4 * 128;
    unsigned char *Ahi = sm, *Alo = Ahi + a_bytes, *Bhi = Alo + a_bytes, *Blo = Bhi + b_bytes;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    __shared__ int timed_out;

    const float *Cs = Cf + (sg ? (size_t)M * na : 0);
    const uint16_t *vl = virt_list + (size_t)w * (2 * M - ne) + (sg ? M - na : 0);
    const float *At = AinvT + (size_t)w * ((size_t)na * na + (size_t)nb * nb) + (sg ? (size_t)na * na : 0);

    // ---- stage the operands (zero K padding; rows beyond nv / n only feed unused outputs)
    for (int t = tid; t < kM * Kp; t += kThreads) {
        const int r = t / Kp, k = t - r * Kp;
        float v = 0.0f;
        if (r < nv && k < n) v = Cs[(size_t)vl[r] * n + k];
        float hi, lo;
        split_tf32(v, hi, lo);
        const uint32_t o = core_off(r, k, kp4);
        *(float *)(Ahi + o) = hi;
        *(float *)(Alo + o) = lo;
    }
    for (int t = tid; t < Np * Kp; t += kThreads) {
        const int r = t / Kp, k = t - r * Kp;
        float v = 0.0f;
        if (r < n && k < n) v = At[(size_t)r * n + k];
        float hi, lo;
        split_tf32(v, hi, lo);
        const uint32_t o = core_off(r, k, kp4);
        *(float *)(Bhi + o) = hi;
        *(float *)(Blo + o) = lo;
    }
    if (tid == 0) {
        timed_out = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {   // allocate 128 columns of tensor memory (N <= 128)
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(smem_u32(&tmem_base)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;");   // generic-proxy stores -> tensor-core reads
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;

    // ---- one thread issues the MMAs: K steps of 8, three products each
    if (tid == 0) {
        const uint32_t idesc = make_idesc(kM, Np);
        // no-swizzle K-major: core matrices along K are 128 B apart, row groups kp4 * 128 B apart
        const uint32_t kstride = 128, rstride = (uint32_t)kp4 * 128;
        const uint32_t lbo = lbo_k_major ? kstride : rstride, sbo = lbo_k_major ? rstride : kstride;
        const uint32_t ah = smem_u32(Ahi), al = smem_u32(Alo), bh = smem_u32(Bhi), bl = smem_u32(Blo);
        for (int ks = 0; ks < Kp / 8; ++ks) {
            const uint32_t koff = (uint32_t)ks * 256;   // two core matrices along K
            const uint64_t dah = make_desc(ah + koff, lbo, sbo), dal = make_desc(al + koff, lbo, sbo);
            const uint64_t dbh = make_desc(bh + koff, lbo, sbo), dbl = make_desc(bl + koff, lbo, sbo);
            const uint32_t acc0 = ks > 0 ? 1u : 0u;
            asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                         "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
                         ::"r"(tmem), "l"(dah), "l"(dbh), "r"(idesc), "r"(acc0));
            asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                         "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
                         ::"r"(tmem), "l"(dah), "l"(dbl), "r"(idesc), "r"(1u));
            asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                         "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
                         ::"r"(tmem), "l"(dal), "l"(dbh), "r"(idesc), "r"(1u));
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     ::"r"(smem_u32(&mbar)));
    }
    // ---- bounded wait for the MMAs
    {
        uint32_t done = 0;
        unsigned spin = 0;
        while (!done && spin < kMaxSpin) {
            asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
                         "selp.u32 %0, 1, 0, p;\n\t}"
                         : "=r"(done) : "r"(smem_u32(&mbar)));
            ++spin;
        }
        if (!done) atomicOr(&timed_out, 1);
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    __syncthreads();
    if (!timed_out) {
        // ---- read D: warp w owns tensor-memory lanes 32w..32w+31 (= rows), 16 columns at a time
        const int row = warp * 32 + lane;
        float *Gw = G + (size_t)w * ((size_t)(M - na) * na + (size_t)(M - nb) * nb) + (sg ? (size_t)(M - na) * na : 0);
        for (int c0 = 0; c0 < Np; c0 += 16) {
            uint32_t r[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                         "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                           "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
                           "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                         : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            if (row < nv) {
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    if (c0 + j < n) Gw[(size_t)row * n + c0 + j] = __uint_as_float(r[j]);
            }
        }
    } else if (tid == 0) {
        atomicOr(status, VMC_DEV_TIMEOUT);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem));
    }
}

}  // namespace

// Returns VMC_ERR_ARG (nothing launched) when the shapes are outside the kernel's range.
vmc_status launch_g_umma(vmc_ctx *ctx, const vmc_walkers *Wk, const float *Cf) {
    const int M = Wk->M, na = Wk->n_alpha, nb = Wk->n_beta;
    const int nmax = na > nb ? na : nb;
    const int nvmax = M - (na < nb ? na : nb);
    if (nmax > 128 || nvmax > kM || nmax < 1) return VMC_ERR_ARG;
    const int Kp = (nmax + 7) & ~7, Np = (nmax + 15) & ~15;
    const size_t smem = (size_t)2 * (kM / 8) * (Kp / 4) * 128 + (size_t)2 * (Np / 8) * (Kp / 4) * 128 + 1024;
    cudaError_t e = cudaFuncSetAttribute(k_g_umma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        k_g_umma<<<dim3(Wk->W, 2), kThreads, smem, ctx->stream>>>(M, na, nb, Cf, Wk->virt_list,
                                                                  (const float *)Wk->AinvT, (float *)Wk->G,
                                                                  ctx->d_status, 1);
    ctx->launches += 1;
    if (e == cudaSuccess) e = cudaGetLastError();
    return cuda_check(ctx, e, "k_g_umma");
}
