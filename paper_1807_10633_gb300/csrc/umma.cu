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
constexpr int kPreChunks = 8;    // k_g_umma: 16-byte chunks per thread held for the next item

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

// The same work split in two halves, for one pass (chunks <= kPre * blockDim.x): the global loads of
// a tile into registers, and later the split into hi/lo tiles in shared memory.  Between the two the
// loads stay in flight, so a persistent kernel can fetch its next item while it works on this one.
template <int kPre>
__device__ __forceinline__ void load_tile_regs(const float *__restrict__ src, int ld, int nrows, int ncols, int Kp,
                                               float4 (&v)[kPre]) {
    const int kp4 = Kp >> 2, rg_n = (nrows + 7) >> 3;
    const int chunks = rg_n * kp4 * 8;
    const bool vec = (ld & 3) == 0 && (((uintptr_t)src) & 15) == 0;
#pragma unroll
    for (int u = 0; u < kPre; ++u) {
        const int e = threadIdx.x + u * blockDim.x;
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
}

template <int kPre>
__device__ __forceinline__ void store_tile_regs(const float4 (&v)[kPre], int nrows, int Kp, unsigned char *hi_t,
                                                unsigned char *lo_t) {
    const int chunks = ((nrows + 7) >> 3) * (Kp >> 2) * 8;
#pragma unroll
    for (int u = 0; u < kPre; ++u) {
        const int e = threadIdx.x + u * blockDim.x;
        if (e < chunks) {
            float4 h, l;
            split_tf32(v[u].x, h.x, l.x); split_tf32(v[u].y, h.y, l.y);
            split_tf32(v[u].z, h.z, l.z); split_tf32(v[u].w, h.w, l.w);
            const uint32_t o = (uint32_t)e * 16;
            *(float4 *)(hi_t + o) = h;
            *(float4 *)(lo_t + o) = l;
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
// kPre > 0 (an item's A tile in at most kPre 16-byte chunks per thread, and M <= kThreads): the
// global loads of item i+1's A tile and orbital map are issued into registers right after item i
// is staged, so their latency overlaps item i's MMAs and item i-1's epilogue.
template <int kPre>
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
    float4 pre[kPre > 0 ? kPre : 1];   // the next item's A tile chunks (kPre > 0)
    uint16_t pre_pos = 0;              // and its orbital-map entry tid
    auto load_item = [&](int t) {
        const int s = t >= W, w = t - s * W, n = s ? nb : na;
        if constexpr (kPre > 0)
            load_tile_regs<kPre>(AinvT + (size_t)w * astride + (s ? (size_t)na * na : 0), n, n, n, Kp, pre);
        pre_pos = tid < M ? pos_all[(size_t)w * 2 * M + (size_t)s * M + tid] : (uint16_t)0;
    };
    if (kPre > 0) load_item(t0);

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
        if constexpr (kPre > 0) {
            store_tile_regs<kPre>(pre, n, Kp, Ah, Al);
            if (tid < M) posb[buf * M + tid] = pre_pos;
            if (t + 1 < t1) load_item(t + 1);
        } else {
            const float *At = AinvT + (size_t)w * astride + (s ? (size_t)na * na : 0);
            stage_tile<8>(At, n, n, n, Kp, Ah, Al);
            const uint16_t *pw = pos_all + (size_t)w * 2 * M + (size_t)s * M;
            for (int k = tid; k < M; k += kThreads) posb[buf * M + k] = pw[k];
        }
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

// ---------------------------------------------------------------------------------------------
// Jastrow block of the walker sums (Sec. III.B: O_pq = n_p n_q) on the tensor cores, exactly.
//
// part[o][c][p][q] = sum over the walkers w of chunk c of cq_o[w] n_w[p] n_w[q]  (p <= q),
// the same 64-bit fixed-point sums as the integer kernel.  The weights are split into eight
// balanced base-256 digits, cq = sum_l d_l 256^l with d_l in [-128, 128), and for every digit
// D_l[p][j] = sum_w n_w[p] (d_l,w n_w[q_j]) is a product of a 0/1 matrix and a small-integer
// matrix: TF32 holds both operands exactly and the FP32 accumulation is exact while every
// partial sum stays below 2^24 (|D_l| <= 128 x walkers per chunk <= 2^23).  The epilogue forms
// sum_l D_l 256^l in 64-bit integers with wrapping arithmetic; the chunk's true sum is below
// 2^62 in magnitude, so the wrapped result is exact.
//
// CTA = (tile, walker chunk).  Tile (P, Q) = spin orbitals p in [128 P, 128 P + 128) (MMA rows) x
// q in [32 Q, 32 Q + 32), for every such block that holds some p <= q (Q >= 4 P).  MMA columns
// j = 256 o + 32 l + q' (weight set o, digit l, q = 32 Q + q'); one or two N = 256 accumulators in
// tensor memory.  Walkers are staged 32 at a time (the K dimension) into double-buffered K-major
// core-matrix tiles.
constexpr int kJB = 32;                 // walkers per K block
constexpr int kJDig = 8;                // base-256 digits of a 64-bit weight
constexpr int kJMaxChunk = 65536;       // walkers per chunk: 128 x 65536 = 2^23 < 2^24
constexpr uint32_t kJA = 128 * kJB * 4; // bytes of the A tile (128 rows)
constexpr uint32_t kJBset = 256 * kJB * 4; // bytes of one weight set's B tile (256 rows)

__host__ __device__ inline int grad_j_tiles(int N2) {
    const int nP = (N2 + 127) / 128, nQ = (N2 + 31) / 32;
    int t = 0;
    for (int P = 0; P < nP; ++P) t += nQ - 4 * P;
    return t;
}

__global__ void __launch_bounds__(kThreads, 1)
k_grad_J_umma(int W, int M, int chunk, const uint32_t *__restrict__ bits, const long long *__restrict__ cq,
              int mode, long long *__restrict__ part, unsigned *status) {
    const int N2 = 2 * M, nw = (M + 31) / 32, nW2 = 2 * nw;
    const int nQ = (N2 + 31) / 32;
    int t = blockIdx.x, P = 0;
    while (t >= nQ - 4 * P) { t -= nQ - 4 * P; ++P; }
    const int Q = 4 * P + t;                       // tiles with 32 Q + 31 >= 128 P
    const int n_sets = mode ? 2 : 1;
    const int c = blockIdx.y, n_chunks = gridDim.y;
    const int w_begin = c * chunk, w_end = min(W, w_begin + chunk);
    const int nblk = w_end > w_begin ? (w_end - w_begin + kJB - 1) / kJB : 0;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *base = (unsigned char *)(((uintptr_t)sm + 1023) & ~(uintptr_t)1023);
    const uint32_t buf_bytes = kJA + (uint32_t)n_sets * kJBset;
    uint32_t *s_bits = (uint32_t *)(base + 2 * buf_bytes);          // [2][kJB][2 nw]
    float *s_dig = (float *)(s_bits + 2 * kJB * 16);                  // [2][set][digit][kJB]
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    const uint32_t ncols = mode ? 512u : 256u;
    if (tid == 0) {
        abort_flag = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&tmem_base)), "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    uint32_t phase = 0u, pending = 0u;   // bit b: mbarrier b's phase parity / a commit not yet awaited

    // occupation bit of spin orbital p (< N2) of block walker wl in the staged words sb
    auto bit = [&](const uint32_t *sb, int wl, int p) -> uint32_t {
        const int s = p >= M, k = p - s * M;
        return (sb[wl * nW2 + s * nw + (k >> 5)] >> (k & 31)) & 1u;
    };

    // the next blocks' occupation words and weights travel in registers: block b + 1 is stored to
    // shared memory and block b + 2 loaded while block b is built, so global latency overlaps
    uint32_t rb[2];
    long long rc;
    auto load_block = [&](int b) {
        const int w0 = w_begin + b * kJB;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int i = tid + u * kThreads, wl = i / nW2, k = i - wl * nW2;
            rb[u] = (b < nblk && i < kJB * nW2 && w0 + wl < w_end) ? bits[(size_t)(w0 + wl) * nW2 + k] : 0u;
        }
        const int wl = tid & (kJB - 1), o = tid / kJB;
        rc = (b < nblk && tid < kJB * n_sets && w0 + wl < w_end) ? cq[(size_t)o * W + w0 + wl] : 0;
    };
    auto store_block = [&](int sb) {
        uint32_t *sbits = s_bits + sb * kJB * 16;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int i = tid + u * kThreads;
            if (i < kJB * nW2) sbits[i] = rb[u];
        }
        if (tid < kJB * n_sets) {
            const int wl = tid & (kJB - 1), o = tid / kJB;
            float *sdig = s_dig + sb * 2 * kJDig * kJB;
            long long x = rc;
#pragma unroll
            for (int l = 0; l < kJDig; ++l) {
                const int d = (int)(signed char)(x & 0xFF);
                sdig[(o * kJDig + l) * kJB + wl] = (float)d;
                x = (x - d) >> 8;
            }
        }
    };
    load_block(0);
    store_block(0);
    load_block(1);
    __syncthreads();

    for (int blk = 0; blk < nblk; ++blk) {
        const int buf = blk & 1, sb = blk & 1;
        if ((pending >> buf) & 1u) {   // the MMAs that last read this buffer (block blk - 2)
            if (!mbar_wait(&mbar[buf], (phase >> buf) & 1u)) abort_flag = 1;
            phase ^= 1u << buf;
            pending &= ~(1u << buf);
        }
        const uint32_t *cur_bits = s_bits + sb * kJB * 16;
        const float *cur_dig = s_dig + sb * 2 * kJDig * kJB;
        unsigned char *At = base + (size_t)buf * buf_bytes, *Bt = At + kJA;
        // A[p][w] = n_w[128 P + p]: 16-byte chunk e = 4 walkers of one row (core-matrix order)
        for (int e = tid; e < 128 * kJB / 4; e += kThreads) {
            const int r8 = e & 7, cm = e >> 3, kc = cm % (kJB / 4), rg = cm / (kJB / 4);
            const int p = P * 128 + rg * 8 + r8;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (p < N2) {
                v.x = (float)bit(cur_bits, kc * 4 + 0, p); v.y = (float)bit(cur_bits, kc * 4 + 1, p);
                v.z = (float)bit(cur_bits, kc * 4 + 2, p); v.w = (float)bit(cur_bits, kc * 4 + 3, p);
            }
            *(float4 *)(At + (uint32_t)e * 16) = v;
        }
        // B[256 o + 32 l + q'][w] = d_l,o[w] n_w[32 Q + q']: lane = q', warp = 4-walker group
        {
            const int q = Q * 32 + lane, kc = warp;
            uint32_t m0 = 0, m1 = 0, m2 = 0, m3 = 0;
            if (q < N2) {
                m0 = 0u - bit(cur_bits, kc * 4 + 0, q); m1 = 0u - bit(cur_bits, kc * 4 + 1, q);
                m2 = 0u - bit(cur_bits, kc * 4 + 2, q); m3 = 0u - bit(cur_bits, kc * 4 + 3, q);
            }
            for (int o = 0; o < n_sets; ++o) {
                unsigned char *Bo = Bt + (size_t)o * kJBset;
#pragma unroll
                for (int l = 0; l < kJDig; ++l) {
                    const uint4 d = *(const uint4 *)(cur_dig + (o * kJDig + l) * kJB + kc * 4);
                    const int row = l * 32 + lane;
                    *(uint4 *)(Bo + core_off(row, kc * 4, kJB / 4)) = make_uint4(d.x & m0, d.y & m1, d.z & m2, d.w & m3);
                }
            }
        }
        store_block(sb ^ 1);     // block blk + 1
        load_block(blk + 2);
        asm volatile("fence.proxy.async.shared::cta;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (abort_flag) break;
        if (tid == 0) {
            const uint32_t idesc = make_idesc(128, 256);
            const uint32_t lbo = 128, sbo = (kJB / 4) * 128;
            const uint32_t a0 = smem_u32(At), b0 = smem_u32(Bt);
            for (int ks = 0; ks < kJB / 8; ++ks) {
                const uint32_t koff = (uint32_t)ks * 256;
                const uint64_t da = make_desc(a0 + koff, lbo, sbo);
                for (int o = 0; o < n_sets; ++o) {
                    const uint64_t db = make_desc(b0 + (uint32_t)o * kJBset + koff, lbo, sbo);
                    const uint32_t acc = tmem + (uint32_t)(o * 256), accum = (blk > 0 || ks > 0) ? 1u : 0u;
                    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
                                 ::"r"(acc), "l"(da), "l"(db), "r"(idesc), "r"(accum));
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         ::"r"(smem_u32(&mbar[buf])));
        }
        pending |= 1u << buf;
    }
    for (int b = 0; b < 2; ++b)
        if ((pending >> b) & 1u) {
            if (!mbar_wait(&mbar[b], (phase >> b) & 1u)) abort_flag = 1;
            phase ^= 1u << b;
        }
    asm volatile("tcgen05.fence::after_thread_sync;");
    __syncthreads();
    if (!abort_flag) {
        // warps 4g..4g+3 drain (set, q half) pairs k = g, g + 2, ...: lane = row of its sub-partition
        const int wq = warp & 3, g = warp >> 2, p = P * 128 + wq * 32 + lane;
        for (int k = g; k < 2 * n_sets; k += 2) {
            const int o = k >> 1, h = k & 1;
            uint64_t acc[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[j] = 0;
            if (nblk > 0) {
#pragma unroll 1
                for (int l = 0; l < kJDig; ++l) {
                    uint32_t r[16];
                    const uint32_t taddr = tmem + ((uint32_t)(wq * 32) << 16) + (uint32_t)(o * 256 + l * 32 + h * 16);
                    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                                   "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                                   "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                                 : "r"(taddr));
                    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        acc[j] += (uint64_t)(long long)__float2ll_rn(__uint_as_float(r[j])) << (8 * l);
                }
            }
            long long *dst = part + ((size_t)o * n_chunks + c) * (size_t)N2 * N2;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int q = Q * 32 + h * 16 + j;
                if (p < N2 && q < N2 && p <= q) dst[(size_t)p * N2 + q] = (long long)acc[j];
            }
        }
    }
    __syncthreads();
    if (abort_flag && tid == 0) atomicOr(status, VMC_DEV_TIMEOUT);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
    }
}

// ---------------------------------------------------------------------------------------------
// FP64-form G = C_v C_occ^-1 on the tensor cores from exact digit products (Sec. III.B, Eq. R).
//
// Every FP64 operand row is scaled by a power of two 2^E (|x| < 2^E over the row) and rounded to a
// 46-bit fixed-point integer q, which is written in six balanced base-256 digits,
//     x = 2^(E-6) sum_i d_i 256^-i  (+ at most 2^(E-47)),   d_i in [-128, 128):
// the digits are the bytes of q + 0x808080808080 minus 128 (that offset adds 128 to every digit
// position; |q| <= 2^46 keeps the sum inside six bytes).  BF16 holds every digit exactly, a digit
// product is an exact 15-bit integer, and the FP32 accumulation of one diagonal
// D_s = sum_{i+j=s} sum_x a_i[c][x] b_j[k][x] stays exact while every partial sum is below 2^24
// (at most 6 pairs x 128 columns x 2^14 = 1.26e7).  The epilogue forms T = sum_s D_s 256^(5-s) in
// 64-bit integers (exact) and G = T 2^(E_c + F_k - 52) with one rounding.  Diagonals s >= 6 are
// dropped: the result differs from the exact product by less than about 2^-43 n of
// 2^(E_c + F_k), against about 2^-53 n for an FP64 dot product.
//
// CTA = persistent over (spin, walker) items.  Per item: the row exponents E_c of C_occ^-T, then
// per tile of at most 80 virtual orbitals, the columns x in chunks of 32 (two K = 16 MMA steps):
// the A digits (C_occ^-T rows, sliced here) and B digits (rows of C gathered from a per-refresh
// digit table) are staged in a double-buffered pair of K-major core-matrix tiles while the one
// issuing thread runs the previous chunk's 21 digit-pair MMAs per K step into six FP32
// accumulators of 80 columns in tensor memory (480 of 512 columns).
constexpr int kOzS = 6;                 // digits per operand, diagonals kept
constexpr int kOzKC = 32;               // columns x per staged chunk
constexpr int kOzN = 80;                // virtual orbitals per tile (accumulator columns)
constexpr int kOzThreads = 512;         // 16 warps: warp w reads tensor-memory lanes 32 (w % 4)
constexpr uint32_t kOzA = 16u * (kOzKC / 8) * 128;     // one A digit tile: 128 rows x 32 columns
constexpr uint32_t kOzB = (kOzN / 8) * (kOzKC / 8) * 128;   // one B digit tile: 80 rows x 32 columns
constexpr uint32_t kOzBuf = kOzS * (kOzA + kOzB);

// Instruction descriptor: D = F32, A = B = BF16, both K-major, N and M.
__device__ __forceinline__ uint32_t make_idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// biased exponent field of x (0 for zero and subnormals)
__device__ __forceinline__ int oz_expo(double x) {
    return (int)((__double_as_longlong(x) >> 52) & 0x7FF);
}

// round(x 2^(46 - E)) + 0x808080808080 for |x| < 2^E (E = the row's largest biased exponent - 1022);
// its bytes, least significant first, are the digits d_5 .. d_0 plus 128.  Subnormals count as zero.
__device__ __forceinline__ unsigned long long oz_fixed(double x, int E) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int ex = (int)((b >> 52) & 0x7FF);
    long long q = 0;
    if (ex != 0) {
        const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
        const int sh = 1075 + E - 46 - ex;            // >= 7 because ex <= E + 1022
        if (sh < 64) {
            const long long r = (long long)((m + (1ull << (sh - 1))) >> sh);
            q = (b >> 63) ? -r : r;
        }
    }
    return (unsigned long long)(q + 0x808080808080ll);
}

// FP32 bit pattern of digit byte k of u (0..5) minus 128: the float 2^23 + byte, less 2^23 + 128
__device__ __forceinline__ uint32_t oz_digit_f32(uint32_t ulo, uint32_t uhi, int k) {
    const uint32_t t = k < 4 ? __byte_perm(ulo, 0x4B000000u, 0x7440u | (uint32_t)k)
                             : __byte_perm(uhi, 0x4B000000u, 0x7440u | (uint32_t)(k - 4));
    return __float_as_uint(__uint_as_float(t) - 8388736.0f);
}

// Six BF16 digit words for the element pair (x0, x1), most significant digit first: word i holds
// digit i of x0 in its low half and of x1 in its high half.
__device__ __forceinline__ void oz_pair(double x0, double x1, int E, uint32_t w[kOzS]) {
    const unsigned long long u0 = oz_fixed(x0, E), u1 = oz_fixed(x1, E);
    const uint32_t a_lo = (uint32_t)u0, a_hi = (uint32_t)(u0 >> 32);
    const uint32_t b_lo = (uint32_t)u1, b_hi = (uint32_t)(u1 >> 32);
#pragma unroll
    for (int i = 0; i < kOzS; ++i)
        w[i] = __byte_perm(oz_digit_f32(a_lo, a_hi, kOzS - 1 - i), oz_digit_f32(b_lo, b_hi, kOzS - 1 - i), 0x7632u);
}

// Digit table of C (both spins): cdig[spin][digit][k][Kp] BF16 (zero for x >= n_sigma) and the
// row exponents cexp[spin][k].  One warp per (spin, orbital), two columns per lane and step.
__global__ void __launch_bounds__(256)
k_c_digits(int M, int na, int nb, int Kp, const double *__restrict__ Ca, const double *__restrict__ Cb,
           uint16_t *__restrict__ cdig, int *__restrict__ cexp) {
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (gw >= 2 * M) return;
    const int s = gw / M, k = gw - s * M, n = s ? nb : na;
    if (n == 0) return;
    const double *row = (s ? Cb : Ca) + (size_t)k * n;
    int mx = 0;
    for (int x = lane; x < n; x += 32) mx = max(mx, oz_expo(row[x]));
    mx = __reduce_max_sync(0xffffffffu, mx);
    const int E = mx - 1022;
    if (lane == 0) cexp[s * M + k] = E;
    for (int x = 2 * lane; x < Kp; x += 64) {
        uint32_t w[kOzS];
        oz_pair(x < n ? row[x] : 0.0, x + 1 < n ? row[x + 1] : 0.0, E, w);
#pragma unroll
        for (int i = 0; i < kOzS; ++i)
            *(uint32_t *)(cdig + (((size_t)s * kOzS + i) * M + k) * Kp + x) = w[i];
    }
}

__global__ void __launch_bounds__(kOzThreads, 1)
k_g_ozaki(int W, int M, int na, int nb, int Kp, const uint16_t *__restrict__ cdig, const int *__restrict__ cexp,
          const uint16_t *__restrict__ virt_all, const double *__restrict__ AinvT, double *__restrict__ G,
          unsigned *status) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *base = (unsigned char *)(((uintptr_t)sm + 1023) & ~(uintptr_t)1023);
    __shared__ int expA[128], expB[VMC_MAX_M];
    __shared__ uint16_t vs[VMC_MAX_M];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    const size_t gstride = (size_t)(M - na) * na + (size_t)(M - nb) * nb;
    const size_t astride = (size_t)na * na + (size_t)nb * nb;
    const size_t vstride = (size_t)2 * M - na - nb;
    const int total = 2 * W, per = (total + gridDim.x - 1) / gridDim.x;
    const int t0 = blockIdx.x * per, t1 = min(total, t0 + per);
    if (t0 >= t1) return;
    if (tid == 0) {
        abort_flag = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&tmem_base)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    uint32_t phase[2] = {0u, 0u};
    bool pending[2] = {false, false};
    int gq = 0;                                    // chunks issued by this CTA
    // wait until the MMAs committed to buffer b have finished
    auto drain = [&](int b) {
        if (!pending[b]) return;
        if (!mbar_wait(&mbar[b], phase[b])) abort_flag = 1;   // every waiter that times out writes 1
        phase[b] ^= 1u;
        pending[b] = false;
    };
    const int nchunks = (Kp + kOzKC - 1) / kOzKC;

    for (int t = t0; t < t1 && !abort_flag; ++t) {
        const int s = t >= W, w = t - s * W, n = s ? nb : na, nv = M - n;
        if (n == 0 || nv == 0) continue;
        const double *At = AinvT + (size_t)w * astride + (s ? (size_t)na * na : 0);
        const uint16_t *vl = virt_all + (size_t)w * vstride + (s ? (size_t)(M - na) : 0);
        double *Gw = G + (size_t)w * gstride + (s ? (size_t)(M - na) * na : 0);
        // row exponents of C_occ^-T: four threads per row, their loads all in flight; the virtual
        // orbitals and their row exponents
        {
            const int c = tid >> 2, part = tid & 3;
            int mx = 0;
            if (c < n) {
#pragma unroll 8
                for (int x = part; x < n; x += 4) mx = max(mx, oz_expo(__ldg(At + (size_t)c * n + x)));
            }
            mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
            mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
            if (c < n && part == 0) expA[c] = mx - 1022;
        }
        for (int v = tid; v < nv; v += kOzThreads) {
            const int k = vl[v];
            vs[v] = (uint16_t)k;
            expB[v] = cexp[s * M + k];
        }
        __syncthreads();
        for (int v0 = 0; v0 < nv && !abort_flag; v0 += kOzN) {
            const int nt = min(kOzN, nv - v0), NP = (nt + 15) & ~15;
            const int nA = ((n + 7) >> 3) * (kOzKC / 8) * 8, nB = ((nt + 7) >> 3) * (kOzKC / 8) * 8;
            for (int q = 0; q < nchunks; ++q, ++gq) {
                const int b = gq & 1;
                drain(b);                              // the MMAs that read this buffer are done
                __syncthreads();                       // abort_flag is uniform after the barrier
                if (abort_flag) break;
                unsigned char *Ab = base + (size_t)b * kOzBuf, *Bb = Ab + kOzS * kOzA;
                const int x0 = q * kOzKC;
                // work item = 8 columns of one row: A digits (rows c < n, sliced here), then B digits
                // (rows v < nt, gathered from the digit table of C); 16 bytes per digit tile each
                for (int e = tid; e < nA + nB; e += kOzThreads) {
                    const bool isA = e < nA;
                    const int ee = isA ? e : e - nA;
                    const int r8 = ee & 7, cm = ee >> 3, kc = cm % (kOzKC / 8), rg = cm / (kOzKC / 8);
                    const int r = rg * 8 + r8, x = x0 + kc * 8;
                    if (isA) {
                        if (r >= n) continue;
                        const double *src = At + (size_t)r * n;
                        double v[8];
#pragma unroll
                        for (int h = 0; h < 8; ++h) v[h] = x + h < n ? __ldg(src + x + h) : 0.0;
                        const int E = expA[r];
                        uint32_t wd[4][kOzS];
#pragma unroll
                        for (int h = 0; h < 4; ++h) oz_pair(v[2 * h], v[2 * h + 1], E, wd[h]);
#pragma unroll
                        for (int i = 0; i < kOzS; ++i)
                            *(uint4 *)(Ab + (size_t)i * kOzA + (size_t)ee * 16) = make_uint4(wd[0][i], wd[1][i], wd[2][i], wd[3][i]);
                    } else {
                        if (r >= nt) continue;
                        uint4 val[kOzS];
#pragma unroll
                        for (int i = 0; i < kOzS; ++i)
                            val[i] = x < Kp ? __ldg((const uint4 *)(cdig + (((size_t)s * kOzS + i) * M + vs[v0 + r]) * Kp + x))
                                            : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
                        for (int i = 0; i < kOzS; ++i) *(uint4 *)(Bb + (size_t)i * kOzB + (size_t)ee * 16) = val[i];
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;");
                asm volatile("tcgen05.fence::before_thread_sync;");
                __syncthreads();
                asm volatile("tcgen05.fence::after_thread_sync;");
                if (tid == 0) {
                    const uint32_t idesc = make_idesc_bf16(kM, NP);
                    const uint32_t lbo = 128, sbo = (kOzKC / 8) * 128;
                    const int ksteps = min(kOzKC, Kp - x0) / 16;
                    for (int ks = 0; ks < ksteps; ++ks)
#pragma unroll
                        for (int d = 0; d < kOzS; ++d)
#pragma unroll
                            for (int i = 0; i <= d; ++i) {
                                const uint64_t da = make_desc(smem_u32(Ab + (size_t)i * kOzA) + ks * 256, lbo, sbo);
                                const uint64_t db = make_desc(smem_u32(Bb + (size_t)(d - i) * kOzB) + ks * 256, lbo, sbo);
                                const uint32_t accf = (q > 0 || ks > 0 || i > 0) ? 1u : 0u;
                                asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                             "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                                             ::"r"(tmem + (uint32_t)(d * kOzN)), "l"(da), "l"(db), "r"(idesc), "r"(accf));
                            }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                                 ::"r"(smem_u32(&mbar[b])));
                }
                pending[b] = true;
            }
            drain(0);
            drain(1);
            asm volatile("tcgen05.fence::after_thread_sync;");
            __syncthreads();
            if (abort_flag) break;
            // epilogue: warp w reads lanes 32 (w % 4) (rows c) and the column blocks of 8 with
            // index = w / 4 modulo 4
            const int c = (warp & 3) * 32 + lane;
            const int Ec = c < n ? expA[c] : 0;
            for (int cb = warp >> 2; cb < NP / 8; cb += kOzThreads / 128) {
                const int col0 = cb * 8;
                uint32_t r[kOzS][8];
#pragma unroll
                for (int d = 0; d < kOzS; ++d) {
                    const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(d * kOzN + col0);
                    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                                 : "=r"(r[d][0]), "=r"(r[d][1]), "=r"(r[d][2]), "=r"(r[d][3]), "=r"(r[d][4]),
                                   "=r"(r[d][5]), "=r"(r[d][6]), "=r"(r[d][7])
                                 : "r"(taddr));
                }
                asm volatile("tcgen05.wait::ld.sync.aligned;");
                if (c < n) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int v = col0 + j;
                        if (v < nt) {
                            long long T = (long long)__float2int_rn(__uint_as_float(r[0][j]));
#pragma unroll
                            for (int d = 1; d < kOzS; ++d) T = T * 256 + (long long)__float2int_rn(__uint_as_float(r[d][j]));
                            const int e2 = Ec + expB[v0 + v] - 52;
                            Gw[(size_t)(v0 + v) * n + c] =
                                (e2 >= -1022 && e2 <= 1023)
                                    ? (double)T * __longlong_as_double((long long)(e2 + 1023) << 52)
                                    : ldexp((double)T, e2);
                        }
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
        }
        __syncthreads();
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

// Walker chunking of the tensor-core Jastrow sums: about one CTA per SM over all tiles, chunks a
// multiple of the K block and at most kJMaxChunk walkers (the exactness bound).
void grad_j_umma_chunks(int W, int M, int nsm, int *chunk, int *n_chunks) {
    const int T = grad_j_tiles(2 * M);
    int nc = nsm / T;
    if (nc < 1) nc = 1;
    const int nblk = (W + kJB - 1) / kJB;
    if (nc > nblk) nc = nblk;
    int ch = ((W + nc - 1) / nc + kJB - 1) / kJB * kJB;
    if (ch > kJMaxChunk) ch = kJMaxChunk;
    if (ch < kJB) ch = kJB;
    *chunk = ch;
    *n_chunks = (W + ch - 1) / ch;
}

size_t grad_j_umma_smem(int mode) {
    const size_t buf = kJA + (size_t)(mode ? 2 : 1) * kJBset;
    return 1024 + 2 * buf + 2 * (sizeof(uint32_t) * kJB * 16 + sizeof(float) * 2 * kJDig * kJB);
}

vmc_status launch_grad_J_umma(vmc_ctx *ctx, int W, int M, const uint32_t *bits, const long long *cq, int mode,
                              long long *part, int chunk, int n_chunks) {
    if (M < 1 || M > 256 || chunk < kJB || chunk > kJMaxChunk || chunk % kJB) return VMC_ERR_ARG;
    const size_t smem = grad_j_umma_smem(mode);
    cudaError_t e = cudaFuncSetAttribute(k_grad_J_umma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        k_grad_J_umma<<<dim3(grad_j_tiles(2 * M), n_chunks), kThreads, smem, ctx->stream>>>(
            W, M, chunk, bits, cq, mode, part, ctx->d_status);
    ctx->launches += 1;
    if (e == cudaSuccess) e = cudaGetLastError();
    return cuda_check(ctx, e, "k_grad_J_umma");
}

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
    // register prefetch of the next item when an A tile fits in kPreChunks 16-byte chunks per thread
    const int nmax = na > nb ? na : nb, Kp = (nmax + 7) & ~7;
    const bool pre = ((nmax + 7) / 8) * (Kp / 4) * 8 <= kPreChunks * kThreads && M <= kThreads;
    const int grid = std::min(nsm, 2 * Wk->W);
    if (pre) {
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_g_umma<kPreChunks>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            k_g_umma<kPreChunks><<<grid, kThreads, smem, ctx->stream>>>(Wk->W, M, na, nb, Cf, Wk->pos,
                                                                        (const float *)Wk->AinvT, (float *)Wk->G,
                                                                        ctx->d_status, 1);
    } else {
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_g_umma<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            k_g_umma<0><<<grid, kThreads, smem, ctx->stream>>>(Wk->W, M, na, nb, Cf, Wk->pos, (const float *)Wk->AinvT,
                                                               (float *)Wk->G, ctx->d_status, 1);
    }
    ctx->launches += 1;
    if (e == cudaSuccess) e = cudaGetLastError();
    return cuda_check(ctx, e, "k_g_umma");
}

// FP64-form G from exact digit products: digit table of C, then the persistent tcgen05 kernel.
bool g_ozaki_ok(int M, int na, int nb) {
    const int nmax = na > nb ? na : nb;
    return nmax >= 1 && nmax <= 128 && M <= VMC_MAX_M;
}

// digit table (2 spins x 6 digits x M rows x Kp BF16, Kp <= M rounded up to 16) + row exponents
size_t g_ozaki_table_bytes(int M) {
    const size_t Kp = (size_t)((M + 15) & ~15);
    return 2 * kOzS * (size_t)M * Kp * sizeof(uint16_t) + 2 * (size_t)M * sizeof(int);
}

vmc_status launch_g_ozaki(vmc_ctx *ctx, const vmc_walkers *Wk, const double *Ca, const double *Cb, void *table) {
    const int M = Wk->M, na = Wk->n_alpha, nb = Wk->n_beta, nmax = na > nb ? na : nb;
    if (!g_ozaki_ok(M, na, nb) || !table) return VMC_ERR_ARG;
    const int Kp = (nmax + 15) & ~15;
    uint16_t *cdig = (uint16_t *)table;
    int *cexp = (int *)(cdig + 2 * kOzS * (size_t)M * Kp);
    k_c_digits<<<(2 * M * 32 + 255) / 256, 256, 0, ctx->stream>>>(M, na, nb, Kp, Ca, Cb, cdig, cexp);
    ctx->launches += 1;
    cudaError_t e = cudaGetLastError();
    int dev = 0, nsm = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = 2 * (size_t)kOzBuf + 1024;
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_g_ozaki, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int grid = std::min(nsm, 2 * Wk->W);
    if (e == cudaSuccess && grid > 0)
        k_g_ozaki<<<grid, kOzThreads, smem, ctx->stream>>>(Wk->W, M, na, nb, Kp, cdig, cexp, Wk->virt_list,
                                                         (const double *)Wk->AinvT, (double *)Wk->G, ctx->d_status);
    ctx->launches += 1;
    if (e == cudaSuccess) e = cudaGetLastError();
    return cuda_check(ctx, e, "k_g_ozaki");
}
