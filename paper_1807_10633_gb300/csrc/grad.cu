// Gradient ratios (Sec. III.B) summed over walkers with per-walker weights (a vector-Jacobian
// product of ln psi), AMSGrad (Sec. II.C, Eqs. m1-m2) and the walker sums of Eq. (vmc).
//
// The walker sums are deterministic: the Jastrow block is an exact 64-bit fixed-point sum, and
// for the orbital block each CTA reduces a fixed chunk of walkers into a partial buffer that a
// second kernel adds in chunk order.
#include <math.h>

#include <algorithm>

#include "common.cuh"

namespace {

constexpr int kChunkJ = 256;    // walkers per CTA for dJ
constexpr int kChunkC = 64;     // walkers per CTA for dC
constexpr int kRowsC = 16;      // orbital rows per CTA (registers per thread) for dC

// 32 consecutive spin-orbital occupation bits starting at spin orbital p0 (lane l -> bit l)
__device__ __forceinline__ uint32_t window_bits(const uint32_t *bits_w, int M, int nw, int p0, int lane) {
    const int p = p0 + lane;
    int bit = 0;
    if (p < 2 * M) {
        const int s = p >= M, k = p - s * M;
        bit = (bits_w[s * nw + (k >> 5)] >> (k & 31)) & 1;
    }
    return __ballot_sync(0xffffffffu, bit);
}

// Weights of walker w: mode 0 -> (t[w]); mode 1 -> (t[w], t[w] e[w]).
__device__ __forceinline__ void weights(int mode, const double *t, const double *e, int w, double &c0, double &c1) {
    c0 = t[w];
    c1 = mode ? c0 * e[w] : 0.0;
}

// Fixed-point weights for the Jastrow gradient: cq = round(c 2^s) with s chosen from sum |c| so that
// no partial sum can overflow 63 bits; integer sums are then exact and order independent.
// Also adds sum c0 and sum c1 to sums[0..1] (mode 1).  Three launches, each sum in a fixed order:
// per-CTA partial sums over consecutive walker chunks, one warp that adds the partials and sets the
// exponents, then the quantisation over the whole grid.
constexpr int kWeightChunk = 256;   // walkers per partial-sum CTA
constexpr int kWeightParts = 256;   // most partial sums (chunks grow beyond 65,536 walkers)

__global__ void __launch_bounds__(256)
k_weight_partial(int W, int chunk, const double *__restrict__ t, const double *__restrict__ e, int mode,
                 double *__restrict__ part) {
    __shared__ double r[4][8];
    double a0 = 0.0, a1 = 0.0, s0 = 0.0, s1 = 0.0;
    const int w0 = blockIdx.x * chunk, w1 = min(W, w0 + chunk);
    for (int w = w0 + threadIdx.x; w < w1; w += blockDim.x) {
        double c0, c1;
        weights(mode, t, e, w, c0, c1);
        a0 += fabs(c0); a1 += fabs(c1); s0 += c0; s1 += c1;
    }
    a0 = warp_sum_f64(a0); a1 = warp_sum_f64(a1); s0 = warp_sum_f64(s0); s1 = warp_sum_f64(s1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { r[0][warp] = a0; r[1][warp] = a1; r[2][warp] = s0; r[3][warp] = s1; }
    __syncthreads();
    if (threadIdx.x < 4) {
        double v = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) v += r[threadIdx.x][k];
        part[(size_t)blockIdx.x * 4 + threadIdx.x] = v;
    }
}

__global__ void __launch_bounds__(32)
k_weight_finish(int n_parts, const double *__restrict__ part, int *__restrict__ sexp, double *__restrict__ sums) {
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < n_parts; b += 32)
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] += part[(size_t)b * 4 + q];
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = warp_sum_f64(v[q]);
    if (threadIdx.x == 0) {
        sexp[0] = v[0] > 0.0 ? 61 - ilogb(v[0]) : 0;
        sexp[1] = v[1] > 0.0 ? 61 - ilogb(v[1]) : 0;
        if (sums) { sums[0] += v[2]; sums[1] += v[3]; }
    }
}

__global__ void __launch_bounds__(256)
k_weight_quant(int W, const double *__restrict__ t, const double *__restrict__ e, int mode,
               const int *__restrict__ sexp, long long *__restrict__ cq) {
    const int e0 = sexp[0], e1 = sexp[1];
    for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < W; w += gridDim.x * blockDim.x) {
        double c0, c1;
        weights(mode, t, e, w, c0, c1);
        cq[w] = __double2ll_rn(scalbn(c0, e0));
        if (mode) cq[W + w] = __double2ll_rn(scalbn(c1, e1));
    }
}

// dJ partials: tile (P, Q) of 32 x 32 spin orbitals with P <= Q, walker chunk blockIdx.y.
// Exact 64-bit integer sums of the fixed-point weights.  part layout: [n_out][chunk][N2][N2].
// The chunk's 32-orbital occupation windows and weights are staged in shared memory; lane l of
// warp v owns p = 32P + l and q = 32Q + 4v .. 4v + 3, so the q bits are warp-uniform (a branch)
// and the p bit is a mask.
__global__ void __launch_bounds__(256)
k_grad_J(int W, int M, const uint32_t *__restrict__ bits, const long long *__restrict__ cq, int mode,
         long long *__restrict__ part) {
    const int N2 = 2 * M, nw = (M + 31) / 32, T = (N2 + 31) / 32;
    int t = blockIdx.x, P = 0;
    while (t >= T - P) { t -= T - P; ++P; }
    const int Q = P + t;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
    __shared__ uint2 s_b[kChunkJ];
    __shared__ longlong2 s_c[kChunkJ];
    const int w0 = blockIdx.y * kChunkJ, nwk = min(W, w0 + kChunkJ) - w0;
    if ((M & 31) == 0) {   // windows are whole words of one spin
        const int wp = P * 32 < M ? P : nw + (P * 32 - M) / 32, wq = Q * 32 < M ? Q : nw + (Q * 32 - M) / 32;
        for (int i = tid; i < nwk; i += blockDim.x) {
            const uint32_t *bw = bits + (size_t)(w0 + i) * 2 * nw;
            s_b[i] = make_uint2(bw[wp], bw[wq]);
        }
    } else {
        for (int i = warp; i < nwk; i += nwarp) {
            const uint32_t *bw = bits + (size_t)(w0 + i) * 2 * nw;
            const uint32_t bp = window_bits(bw, M, nw, P * 32, lane);
            const uint32_t bq = window_bits(bw, M, nw, Q * 32, lane);
            if (lane == 0) s_b[i] = make_uint2(bp, bq);
        }
    }
    for (int i = tid; i < nwk; i += blockDim.x) {
        longlong2 c;
        c.x = cq[w0 + i];
        c.y = mode ? cq[W + w0 + i] : 0;
        s_c[i] = c;
    }
    __syncthreads();
    const int qb = warp * 4;
    long long acc[4] = {0, 0, 0, 0}, acc2[4] = {0, 0, 0, 0};
    if (mode) {
        for (int i = 0; i < nwk; ++i) {
            const uint2 b = s_b[i];
            const longlong2 c = s_c[i];
            const long long m = -(long long)((b.x >> lane) & 1u);
            const long long c0 = c.x & m, c1 = c.y & m;
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if ((b.y >> (qb + k)) & 1u) { acc[k] += c0; acc2[k] += c1; }
        }
    } else {
        for (int i = 0; i < nwk; ++i) {
            const uint2 b = s_b[i];
            const long long c0 = s_c[i].x & -(long long)((b.x >> lane) & 1u);
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if ((b.y >> (qb + k)) & 1u) acc[k] += c0;
        }
    }
    const size_t chunk_sz = (size_t)N2 * N2;
    long long *dst = part + (size_t)blockIdx.y * chunk_sz;
    long long *dst2 = part + ((size_t)gridDim.y + blockIdx.y) * chunk_sz;
    const int p = P * 32 + lane;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int q = Q * 32 + qb + k;
        if (p < N2 && q < N2 && p <= q) {
            dst[(size_t)p * N2 + q] = acc[k];
            if (mode) dst2[(size_t)p * N2 + q] = acc2[k];
        }
    }
}

__global__ void k_reduce_J(int M, int n_chunks, const long long *__restrict__ part, const int *__restrict__ sexp,
                           double *__restrict__ dJ, double *__restrict__ dJ2) {
    const int N2 = 2 * M;
    const size_t csz = (size_t)N2 * N2;
    const int e0 = sexp[0], e1 = sexp[1];
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < N2 * N2; t += gridDim.x * blockDim.x) {
        const int p = t / N2, q = t % N2;
        if (p > q) continue;
        long long s = 0, s2 = 0;
        for (int c = 0; c < n_chunks; ++c) s += part[(size_t)c * csz + t];
        dJ[t] += scalbn((double)s, -e0);
        if (dJ2) {
            for (int c = 0; c < n_chunks; ++c) s2 += part[((size_t)n_chunks + c) * csz + t];
            dJ2[t] += scalbn((double)s2, -e1);
        }
    }
}

// dC partials: CTA = (spin, block of kRowsC orbital rows) x walker chunk; thread x owns the
// accumulators dC[k][x] of its rows in registers: acc[k][x] += c_w AinvT_w[pos_w(k)][x] for
// occupied k.  part layout: [n_out][chunk][2][M][nmax].  acc_t = float (mixed) or double.
template <typename real, typename acc_t>
__global__ void __launch_bounds__(128)
k_grad_C(int W, int M, int na, int nb, const uint16_t *__restrict__ pos, const real *__restrict__ AinvT,
         const double *__restrict__ wgt, const double *__restrict__ e, int mode, double *__restrict__ part) {
    const int nrb = (M + kRowsC - 1) / kRowsC;
    const int s = blockIdx.x / nrb, rb = blockIdx.x - s * nrb;
    const int n = s ? nb : na, x = threadIdx.x;
    const int k0 = rb * kRowsC;
    acc_t acc[kRowsC], acc2[kRowsC];
#pragma unroll
    for (int r = 0; r < kRowsC; ++r) { acc[r] = 0; acc2[r] = 0; }
    const size_t astride = (size_t)na * na + (size_t)nb * nb;
    const size_t aoff = s ? (size_t)na * na : 0;
    const int w0 = blockIdx.y * kChunkC, w1 = min(W, w0 + kChunkC);
    const bool xin = x < n;
    // the kRowsC map entries of a walker: two 16-byte loads when aligned (M % 8 == 0)
    const bool vec = (M & 7) == 0 && k0 + kRowsC <= M;
    auto map_of = [&](int w, uint4 &lo, uint4 &hi) {
        const uint16_t *pw = pos + (size_t)w * 2 * M + (size_t)s * M + k0;
        if (vec) {
            lo = __ldg((const uint4 *)pw);
            hi = __ldg((const uint4 *)pw + 1);
        } else {
            uint16_t t[kRowsC];
#pragma unroll
            for (int r = 0; r < kRowsC; ++r) t[r] = k0 + r < M ? pw[r] : (uint16_t)0x8000;
            uint32_t q[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) q[k] = (uint32_t)t[2 * k] | ((uint32_t)t[2 * k + 1] << 16);
            lo = make_uint4(q[0], q[1], q[2], q[3]);
            hi = make_uint4(q[4], q[5], q[6], q[7]);
        }
    };
    uint4 nlo = make_uint4(0, 0, 0, 0), nhi = nlo;
    if (w0 < w1) map_of(w0, nlo, nhi);
    for (int w = w0; w < w1; ++w) {
        const uint4 lo = nlo, hi = nhi;
        if (w + 1 < w1) map_of(w + 1, nlo, nhi);    // prefetch the next walker's map
        double c0d, c1d;
        weights(mode, wgt, e, w, c0d, c1d);
        const acc_t c0 = (acc_t)c0d, c1 = (acc_t)c1d;
        const real *A = AinvT + (size_t)w * astride + aoff;
        const uint32_t words[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
        real a[kRowsC];
#pragma unroll
        for (int r = 0; r < kRowsC; ++r) {         // all row loads in flight together
            const uint32_t pc = (words[r >> 1] >> ((r & 1) * 16)) & 0xFFFFu;
            a[r] = (xin && k0 + r < M && !(pc & 0x8000u)) ? A[(size_t)pc * n + x] : real(0);
        }
#pragma unroll
        for (int r = 0; r < kRowsC; ++r) {
            acc[r] += c0 * (acc_t)a[r];
            if (mode) acc2[r] += c1 * (acc_t)a[r];
        }
    }
    if (!xin) return;
    const size_t blk = (size_t)M * (na > nb ? na : nb);
    double *dst = part + ((size_t)blockIdx.y * 2 + s) * blk;
    double *dst2 = part + (((size_t)gridDim.y + blockIdx.y) * 2 + s) * blk;
#pragma unroll
    for (int r = 0; r < kRowsC; ++r) {
        const int k = k0 + r;
        if (k >= M) break;
        dst[(size_t)k * n + x] = (double)acc[r];
        if (mode) dst2[(size_t)k * n + x] = (double)acc2[r];
    }
}

// Sum of the dC partials over walker chunks.  CTA = 32 consecutive outputs (lanes, coalesced) x 8
// warps; warp v adds chunks v, v + 8, ... into four running sums (more loads in flight), then the
// eight warp sums are added in warp order: a fixed order, so the result is deterministic.
__global__ void __launch_bounds__(256)
k_reduce_C(int M, int na, int nb, int n_chunks, int n_out, const double *__restrict__ part,
           double *__restrict__ dCa, double *__restrict__ dCb, double *__restrict__ dCa2, double *__restrict__ dCb2) {
    __shared__ double red[8][33];
    const int nmax = na > nb ? na : nb;
    const int tot = M * na + M * nb, total = n_out * tot;
    const int lane = threadIdx.x & 31, v = threadIdx.x >> 5;
    const int t = blockIdx.x * 32 + lane;
    const int o = t / tot, r = t - o * tot;
    const int s = r >= M * na;
    const int u = s ? r - M * na : r;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    if (t < total) {
        const size_t mn = (size_t)M * nmax, stride = 2 * mn;
        const double *src = part + ((size_t)o * n_chunks * 2 + s) * mn + u;
        int c = v;
        for (; c + 24 < n_chunks; c += 32) {
            acc[0] += src[(size_t)c * stride];
            acc[1] += src[(size_t)(c + 8) * stride];
            acc[2] += src[(size_t)(c + 16) * stride];
            acc[3] += src[(size_t)(c + 24) * stride];
        }
        if (c < n_chunks) acc[0] += src[(size_t)c * stride];            // at most three left
        if (c + 8 < n_chunks) acc[1] += src[(size_t)(c + 8) * stride];
        if (c + 16 < n_chunks) acc[2] += src[(size_t)(c + 16) * stride];
    }
    red[v][lane] = (acc[0] + acc[1]) + (acc[2] + acc[3]);
    __syncthreads();
    if (v == 0 && t < total) {
        double sum = 0.0;
#pragma unroll
        for (int k = 0; k < 8; ++k) sum += red[k][lane];
        double *dst = o == 0 ? (s ? dCb : dCa) : (s ? dCb2 : dCa2);
        dst[u] += sum;
    }
}

__global__ void k_amsgrad(double *p, const double *g, double *m, double *v, size_t np, double alpha,
                          double b1, double b2) {
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < np; k += (size_t)gridDim.x * blockDim.x) {
        const double gk = g[k];
        const double mk = (1.0 - b1) * m[k] + b1 * gk;
        const double cand = (1.0 - b2) * v[k] + b2 * (gk * gk);
        const double vk = v[k] > cand ? v[k] : cand;
        m[k] = mk;
        v[k] = vk;
        if (vk > 0.0) p[k] -= alpha * mk / sqrt(vk);
    }
}

__global__ void k_energy_gradient(size_t n, const double *__restrict__ sums, const double *__restrict__ aO,
                                  const double *__restrict__ aEO, double *__restrict__ g) {
    const double T = sums[0], E = sums[1] / T;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        g[k] = 2.0 * (aEO[k] / T - E * (aO[k] / T));
}

__global__ void __launch_bounds__(1024)
k_walker_reduce(int W, const double *__restrict__ t, const double *__restrict__ e, double *out) {
    __shared__ double r0[32], r1[32];
    double a = 0.0, b = 0.0;
    for (int w = threadIdx.x; w < W; w += blockDim.x) {
        a += t[w];
        b += t[w] * e[w];
    }
    a = warp_sum_f64(a);
    b = warp_sum_f64(b);
    if ((threadIdx.x & 31) == 0) { r0[threadIdx.x >> 5] = a; r1[threadIdx.x >> 5] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sa = 0.0, sb = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { sa += r0[k]; sb += r1[k]; }
        out[0] += sa;
        out[1] += sb;
    }
}

}  // namespace

static vmc_status grad_impl(vmc_ctx *ctx, const vmc_walkers *Wk, const double *t, const double *e, int mode,
                            double *const out0[3], double *const out1[3], double *sums) {
    const int W = Wk->W, M = Wk->M, na = Wk->n_alpha, nb = Wk->n_beta, N2 = 2 * M;
    const int T = (N2 + 31) / 32, ntile = T * (T + 1) / 2;
    const int cc = (W + kChunkC - 1) / kChunkC;
    const bool jtc = ctx->grad_j_tc != 0 && out0[0] != nullptr;
    int cj = (W + kChunkJ - 1) / kChunkJ, chunk_j = kChunkJ;
    if (jtc) {
        int dev = 0, nsm = 0;
        cudaError_t err = cudaGetDevice(&dev);
        if (err == cudaSuccess) err = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (err != cudaSuccess) return cuda_check(ctx, err, "device attributes");
        grad_j_umma_chunks(W, M, nsm, &chunk_j, &cj);
    }
    const int nmax = na > nb ? na : nb, nout = mode + 1;
    if (nmax > 128) return set_err(ctx, VMC_ERR_ARG, "n_sigma > 128 is not supported by the gradient kernel");
    // workspace: [exponents | pad to 256] [partial weight sums] [cq: 2 W int64] [gradient partials]
    const size_t parts = 256 + sizeof(double) * 4 * kWeightParts;
    const size_t head = parts + sizeof(long long) * 2 * (size_t)W;
    const size_t bytes_J = sizeof(long long) * (size_t)nout * cj * N2 * N2;
    const size_t bytes_C = sizeof(double) * (size_t)nout * cc * 2 * M * nmax;
    vmc_status st = ensure_workspace(ctx, head + (bytes_J > bytes_C ? bytes_J : bytes_C));
    if (st) return st;
    int *sexp = (int *)ctx->ws;
    double *wpart = (double *)((char *)ctx->ws + 256);
    long long *cq = (long long *)((char *)ctx->ws + parts);
    void *part = (char *)ctx->ws + head;
    {
        const int wchunk = std::max(kWeightChunk, (W + kWeightParts - 1) / kWeightParts);
        const int n_parts = (W + wchunk - 1) / wchunk;
        k_weight_partial<<<n_parts, 256, 0, ctx->stream>>>(W, wchunk, t, e, mode, wpart);
        k_weight_finish<<<1, 32, 0, ctx->stream>>>(n_parts, wpart, sexp, sums);
        k_weight_quant<<<(W + 255) / 256 < 1216 ? (W + 255) / 256 : 1216, 256, 0, ctx->stream>>>(W, t, e, mode, sexp, cq);
        ctx->launches += 3;
    }
    if (out0[0]) {
        if (jtc) {
            st = launch_grad_J_umma(ctx, W, M, Wk->occ_bits, cq, mode, (long long *)part, chunk_j, cj);
            if (st) return st;     // (the launch is counted there)
        } else {
            k_grad_J<<<dim3(ntile, cj), 256, 0, ctx->stream>>>(W, M, Wk->occ_bits, cq, mode, (long long *)part);
            ctx->launches += 1;
        }
        k_reduce_J<<<(N2 * N2 + 255) / 256, 256, 0, ctx->stream>>>(M, cj, (const long long *)part, sexp, out0[0],
                                                                   mode ? out1[0] : nullptr);
        ctx->launches += 1;
        cudaError_t err = cudaGetLastError();
        if (err != cudaSuccess) return cuda_check(ctx, err, "k_grad_J");
    }
    if (out0[1] && out0[2]) {
        const int nrb = (M + kRowsC - 1) / kRowsC;
        const int threads = ((nmax + 31) / 32) * 32;
        dim3 grid(2 * nrb, cc);
        if (Wk->precision == VMC_FP64)
            k_grad_C<double, double><<<grid, threads, 0, ctx->stream>>>(W, M, na, nb, Wk->pos, (const double *)Wk->AinvT,
                                                                        t, e, mode, (double *)part);
        else
            k_grad_C<float, float><<<grid, threads, 0, ctx->stream>>>(W, M, na, nb, Wk->pos, (const float *)Wk->AinvT,
                                                                      t, e, mode, (double *)part);
        const int tot = nout * (M * na + M * nb);
        k_reduce_C<<<(tot + 31) / 32, 256, 0, ctx->stream>>>(M, na, nb, cc, nout, (const double *)part, out0[1],
                                                               out0[2], mode ? out1[1] : nullptr, mode ? out1[2] : nullptr);
        ctx->launches += 2;
        cudaError_t err = cudaGetLastError();
        if (err != cudaSuccess) return cuda_check(ctx, err, "k_grad_C");
    }
    return VMC_OK;
}

vmc_status launch_grad(vmc_ctx *ctx, const vmc_walkers *Wk, const double *w, double *dJ, double *dCa,
                       double *dCb) {
    double *const o0[3] = {dJ, dCa, dCb};
    double *const o1[3] = {nullptr, nullptr, nullptr};
    return grad_impl(ctx, Wk, w, nullptr, 0, o0, o1, nullptr);
}

vmc_status launch_accumulate(vmc_ctx *ctx, const vmc_walkers *Wk, const double *t, const double *e,
                             double *const aO[3], double *const aEO[3], double *sums) {
    return grad_impl(ctx, Wk, t, e, 1, aO, aEO, sums);
}

vmc_status launch_amsgrad(vmc_ctx *ctx, double *p, const double *g, double *m, double *n, size_t np,
                          double alpha, double b1, double b2) {
    if (np == 0) return VMC_OK;
    const int blocks = (int)((np + 255) / 256 < 152 * 8 ? (np + 255) / 256 : 152 * 8);
    k_amsgrad<<<blocks, 256, 0, ctx->stream>>>(p, g, m, n, np, alpha, b1, b2);
    ctx->launches += 1;
    return cuda_check(ctx, cudaGetLastError(), "k_amsgrad");
}

vmc_status launch_energy_gradient(vmc_ctx *ctx, size_t n, const double *sums, const double *aO,
                                  const double *aEO, double *g) {
    if (n == 0) return VMC_OK;
    const int blocks = (int)((n + 255) / 256 < 152 * 8 ? (n + 255) / 256 : 152 * 8);
    k_energy_gradient<<<blocks, 256, 0, ctx->stream>>>(n, sums, aO, aEO, g);
    ctx->launches += 1;
    return cuda_check(ctx, cudaGetLastError(), "k_energy_gradient");
}

vmc_status launch_walker_reduce(vmc_ctx *ctx, int W, const double *t, const double *e, double *out) {
    k_walker_reduce<<<1, 1024, 0, ctx->stream>>>(W, t, e, out);
    ctx->launches += 1;
    return cuda_check(ctx, cudaGetLastError(), "k_walker_reduce");
}
