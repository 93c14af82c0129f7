// G = C_v C_occ^-1 on the 5th-generation tensor cores (tcgen05, TF32) with a split-precision
// correction, for the mixed-form refresh of the walker tables (Sec. III.B, Eq. R).
//
// Products are split: D = A_hi B_hi + A_hi B_lo + A_lo B_hi (x_hi = x truncated to TF32,
// x_lo = x - x_hi), accumulated in FP32 in tensor memory, which recovers ~22 bits from TF32
// products.  Operands are staged in shared memory in the no-swizzle K-major core-matrix layout
// (8 rows x 16 bytes per core matrix); one thread issues the MMAs and commits them to an
// mbarrier whose waits are bounded (on timeout the kernel latches VMC_ERR_TIMEOUT, frees its
// tensor memory and returns).
#include <stdint.h>

#include <algorithm>

#include "common.cuh"

namespace {

constexpr int kM = 128;          // MMA rows (virtual slots, padded)
constexpr int kThreads = 256;    // eight warps: warp w reads tensor-memory lanes 32 (w % 4)
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

// Stages rows [0, nrows) x K [0, Kp) of a row-major FP32 matrix (leading dimension ld, valid
// columns [0, ncols), zeros beyond) into hi/lo tiles in the K-major no-swizzle core layout.
// Work item = one 16-byte chunk (4 K values of one row); consecutive threads take the 8 rows of a
// core matrix, then the next core matrix along K, so a warp writes 512 contiguous bytes.
template <int kUnroll>
__device__ __forceinline__ void stage_tile(const float *__restrict__ src, int ld, int nrows, int ncols, int Kp,
                                           unsigned char *hi_t, unsigned char *lo_t) {
    const int kp4 = Kp >> 2, rg_n = (nrows + 7) >> 3;
    const int chunks = rg_n * kp4 * 8;
    const bool vec = (ld & 3) == 0 && (((uintptr_t)src) & 15) == 0;
    for (int base = threadIdx.x; base < chunks; base += kUnroll * blockDim.x) {
        float4 v[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int e = base + u * blockDim.x;
            v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (e < chunks) {
                const int r8 = e & 7, cm = e >> 3, kc = cm % kp4, rg = cm / kp4;
                const int row = rg * 8 + r8, k = kc * 4;
                if (row < nrows) {
                    if (vec && k + 3 < ncols) {
                        v[u] = __ldg((const float4 *)(src + (size_t)row * ld + k));
                    } else {
                        float t[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) t[q] = (k + q < ncols) ? src[(size_t)row * ld + k + q] : 0.f;
                        v[u] = make_float4(t[0], t[1], t[2], t[3]);
                    }
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int e = base + u * blockDim.x;
            if (e < chunks) {
                float4 h, l;
                split_tf32(v[u].x, h.x, l.x); split_tf32(v[u].y, h.y, l.y);
                split_tf32(v[u].z, h.z, l.z); split_tf32(v[u].w, h.w, l.w);
                const uint32_t o = (uint32_t)e * 16;   // = core_off(row, k) for this chunk order
                *(float4 *)(hi_t + o) = h;
                *(float4 *)(lo_t + o) = l;
            }
        }
    }
}

// Bounded wait on an mbarrier phase; returns false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity) {
    uint32_t done = 0;
    for (unsigned spin = 0; spin < kMaxSpin && !done; ++spin)
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done) : "r"(smem_u32(mbar)), "r"(parity));
    return done != 0;
}

// Persistent, pipelined G refresh.  Items are (spin, walker) pairs; CTA b takes a contiguous range.
//   MMA operand A (M = 128 >= n rows): AinvT[c][x] of the item's walker and spin (K-major);
//   MMA operand B (N = M_orb rounded up to 16): C^sigma[k][x] for every orbital k, staged once
//   per spin and shared by all items of the CTA;
//   D[c][k] = sum_x AinvT[c][x] C[k][x] = G_full[k][c]; the epilogue keeps the virtual rows k.
// A and the tensor-memory accumulator are double buffered: staging item i+1 and draining item i-1
// overlap the MMAs of item i.  Rows n..127 of the A tile are never written: they read whatever
// follows in shared memory and only feed output rows that are discarded.
__global__ void __launch_bounds__(kThreads, 1)
k_g_umma(int W, int M, int na, int nb, const float *__restrict__ Cf, const uint16_t *__restrict__ pos_all,
         const float *__restrict__ AinvT, float *__restrict__ G, unsigned *status, int lbo_k_major) {
    const int nmax = na > nb ? na : nb;
    const int Kp = (nmax + 7) & ~7, kp4 = Kp >> 2, Mp = (M + 15) & ~15;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    extern __shared__ __align__(1024) unsigned char sm[];
    const uint32_t a_bytes = (uint32_t)((nmax + 7) / 8) * kp4 * 128, b_bytes = (uint32_t)(Mp / 8) * kp4 * 128;
    unsigned char *Abuf = sm;                                  // [2 buffers][hi, lo] of a_bytes
    unsigned char *Bh = sm + 4 * a_bytes, *Bl = Bh + b_bytes;  // C^sigma hi / lo
    uint16_t *posb = (uint16_t *)(Bl + b_bytes);               // [2][M] orbital map of the item
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    const size_t gstride = (size_t)(M - na) * na + (size_t)(M - nb) * nb;
    const size_t astride = (size_t)na * na + (size_t)nb * nb;
    const int total = 2 * W, per = (total + gridDim.x - 1) / gridDim.x;
    const int t0 = blockIdx.x * per, t1 = min(total, t0 + per);
    if (t0 >= t1) return;
    if (tid == 0) {
        abort_flag = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {   // two accumulators of Mp <= 256 columns
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&tmem_base)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    uint32_t phase[2] = {0u, 0u};
    int cur_spin = -1, prev = -1, prev_buf = 0, it = 0;

    // epilogue of item q (accumulator buffer bq): G[w][slot(k)][c] = D[c][k] for virtual k
    auto epilogue = [&](int q, int bq) {
        const int s = q >= W, w = q - s * W, n = s ? nb : na;
        float *Gw = G + (size_t)w * gstride + (s ? (size_t)(M - na) * na : 0);
        const uint16_t *pq = posb + bq * M;
        const int wq = warp & 3, half = warp >> 2;
        const int c = wq * 32 + lane;
        const int nchunk = Mp / 16, ch0 = half ? (nchunk + 1) / 2 : 0, ch1 = half ? nchunk : (nchunk + 1) / 2;
        for (int k0 = ch0 * 16; k0 < ch1 * 16; k0 += 16) {
            uint32_t r[16];
            const uint32_t taddr = tmem + (uint32_t)(bq * 256) + ((uint32_t)(wq * 32) << 16) + (uint32_t)k0;
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                         "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                           "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
                           "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                         : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            if (c < n) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int k = k0 + j;
                    if (k < M) {
                        const uint16_t pk = pq[k];
                        if (pk & 0x8000) Gw[(size_t)(pk & 0x7FFF) * n + c] = __uint_as_float(r[j]);
                    }
                }
            }
        }
    };

    for (int t = t0; t < t1 && !abort_flag; ++t, ++it) {
        const int s = t >= W, w = t - s * W, n = s ? nb : na;
        const int buf = it & 1;
        if (s != cur_spin) {   // (re)stage C^sigma after draining the pipeline
            if (prev >= 0) {
                if (!mbar_wait(&mbar[prev_buf], phase[prev_buf])) { if (tid == 0) abort_flag = 1; }
                phase[prev_buf] ^= 1u;
                asm volatile("tcgen05.fence::after_thread_sync;");
                __syncthreads();
                if (abort_flag) break;
                epilogue(prev, prev_buf);
                prev = -1;
                asm volatile("tcgen05.fence::before_thread_sync;");
                __syncthreads();
            }
            const float *Cs = Cf + (s ? (size_t)M * na : 0);
            stage_tile<2>(Cs, n, M, n, Kp, Bh, Bl);   // also zeroes rows M..ceil8(M)-1
            const int M8 = (M + 7) & ~7;
            for (int e = tid; e < (Mp - M8) * Kp; e += kThreads) {   // zero rows ceil8(M)..Mp-1
                const int r = M8 + e / Kp, k = e % Kp;
                *(float *)(Bh + core_off(r, k, kp4)) = 0.f;
                *(float *)(Bl + core_off(r, k, kp4)) = 0.f;
            }
            cur_spin = s;
        }
        // stage A = AinvT of item t into buffer `buf`, and its orbital map
        unsigned char *Ah = Abuf + (size_t)(2 * buf) * a_bytes, *Al = Ah + a_bytes;
        const float *At = AinvT + (size_t)w * astride + (s ? (size_t)na * na : 0);
        stage_tile<8>(At, n, n, n, Kp, Ah, Al);
        const uint16_t *pw = pos_all + (size_t)w * 2 * M + (size_t)s * M;
        for (int k = tid; k < M; k += kThreads) posb[buf * M + k] = pw[k];
        asm volatile("fence.proxy.async.shared::cta;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (tid == 0) {
            const uint32_t idesc = make_idesc(kM, Mp);
            const uint32_t kstride = 128, ra = (uint32_t)kp4 * 128;
            const uint32_t lbo = lbo_k_major ? kstride : ra, sbo = lbo_k_major ? ra : kstride;
            const uint32_t ah = smem_u32(Ah), al = smem_u32(Al), bh = smem_u32(Bh), bl = smem_u32(Bl);
            const uint32_t acc = tmem + (uint32_t)(buf * 256);
            for (int ks = 0; ks < Kp / 8; ++ks) {
                const uint32_t koff = (uint32_t)ks * 256;
                const uint64_t dah = make_desc(ah + koff, lbo, sbo), dal = make_desc(al + koff, lbo, sbo);
                const uint64_t dbh = make_desc(bh + koff, lbo, sbo), dbl = make_desc(bl + koff, lbo, sbo);
                const uint32_t acc0 = ks > 0 ? 1u : 0u;
                asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                             "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
                             ::"r"(acc), "l"(dah), "l"(dbh), "r"(idesc), "r"(acc0));
                asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                             "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
                             ::"r"(acc), "l"(dah), "l"(dbl), "r"(idesc), "r"(1u));
                asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                             "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
                             ::"r"(acc), "l"(dal), "l"(dbh), "r"(idesc), "r"(1u));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         ::"r"(smem_u32(&mbar[buf])));
        }
        // drain the previous item while these MMAs run
        if (prev >= 0) {
            if (!mbar_wait(&mbar[prev_buf], phase[prev_buf])) { if (tid == 0) abort_flag = 1; }
            phase[prev_buf] ^= 1u;
            asm volatile("tcgen05.fence::after_thread_sync;");
            __syncthreads();
            if (abort_flag) break;
            epilogue(prev, prev_buf);
        }
        prev = t;
        prev_buf = buf;
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
    }
    if (prev >= 0 && !abort_flag) {
        if (!mbar_wait(&mbar[prev_buf], phase[prev_buf])) { if (tid == 0) abort_flag = 1; }
        asm volatile("tcgen05.fence::after_thread_sync;");
        __syncthreads();
        if (!abort_flag) epilogue(prev, prev_buf);
    }
    __syncthreads();
    if (abort_flag && tid == 0) atomicOr(status, VMC_DEV_TIMEOUT);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
    }
}

}  // namespace

// Shared memory of the persistent G kernel, or 0 when the shapes are outside its range.
size_t g_umma_smem(int M, int na, int nb) {
    const int nmax = na > nb ? na : nb;
    if (nmax < 1 || nmax > 128 || M > 256) return 0;
    const int Kp = (nmax + 7) & ~7, Mp = (M + 15) & ~15;
    const size_t a = (size_t)((nmax + 7) / 8) * (Kp / 4) * 128, b = (size_t)(Mp / 8) * (Kp / 4) * 128;
    // the MMA reads 128 rows (16 row groups) from the start of every A buffer, the last one included
    const size_t tile = (size_t)16 * (Kp / 4) * 128;
    const size_t bytes = std::max(4 * a + 2 * b + 2 * 2 * (size_t)M, 3 * a + tile) + 1024;
    return bytes <= 220 * 1024 ? bytes : 0;
}

vmc_status launch_g_umma(vmc_ctx *ctx, const vmc_walkers *Wk, const float *Cf) {
    const int M = Wk->M, na = Wk->n_alpha, nb = Wk->n_beta;
    const size_t smem = g_umma_smem(M, na, nb);
    if (!smem) return VMC_ERR_ARG;
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_g_umma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int grid = std::min(nsm, 2 * Wk->W);
    if (e == cudaSuccess)
        k_g_umma<<<grid, kThreads, smem, ctx->stream>>>(Wk->W, M, na, nb, Cf, Wk->pos, (const float *)Wk->AinvT,
                                                        (float *)Wk->G, ctx->d_status, 1);
    ctx->launches += 1;
    if (e == cudaSuccess) e = cudaGetLastError();
    return cuda_check(ctx, e, "k_g_umma");
}
