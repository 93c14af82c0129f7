// Gradient ratios (Sec. III.B) summed over walkers with per-walker weights (a vector-Jacobian
// product of ln psi), AMSGrad (Sec. II.C, Eqs. m1-m2) and the walker sums of Eq. (vmc).
//
// The walker sums are deterministic: each CTA reduces a fixed chunk of walkers into a partial
// buffer and a second kernel adds the partials in chunk order.
#include <math.h>

#include "common.cuh"

namespace {

constexpr int kChunkJ = 1024;   // walkers per CTA for dJ
constexpr int kChunkC = 256;    // walkers per CTA for dC

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

// dJ partials: tile (P, Q) of 32 x 32 spin orbitals with P <= Q, walker chunk blockIdx.y.
__global__ void __launch_bounds__(256)
k_grad_J(int W, int M, const uint32_t *__restrict__ bits, const double *__restrict__ wgt,
         double *__restrict__ part) {
    const int N2 = 2 * M, nw = (M + 31) / 32, T = (N2 + 31) / 32;
    int t = blockIdx.x, P = 0;
    while (t >= T - P) { t -= T - P; ++P; }
    const int Q = P + t;
    const int tid = threadIdx.x, lane = tid & 31;
    const int pl = tid >> 3, ql0 = (tid & 7) * 4;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    const int w0 = blockIdx.y * kChunkJ, w1 = min(W, w0 + kChunkJ);
    for (int w = w0; w < w1; ++w) {
        const uint32_t *bw = bits + (size_t)w * 2 * nw;
        const uint32_t bp = window_bits(bw, M, nw, P * 32, lane);
        const uint32_t bq = window_bits(bw, M, nw, Q * 32, lane);
        if ((bp >> pl) & 1u) {
            const double c = wgt[w];
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if ((bq >> (ql0 + k)) & 1u) acc[k] += c;
        }
    }
    double *dst = part + (size_t)blockIdx.y * N2 * N2;
    const int p = P * 32 + pl;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int q = Q * 32 + ql0 + k;
        if (p < N2 && q < N2 && p <= q) dst[(size_t)p * N2 + q] = acc[k];
    }
}

__global__ void k_reduce_J(int M, int n_chunks, const double *__restrict__ part, double *__restrict__ dJ) {
    const int N2 = 2 * M;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < N2 * N2; t += gridDim.x * blockDim.x) {
        const int p = t / N2, q = t % N2;
        if (p > q) continue;
        double s = 0.0;
        for (int c = 0; c < n_chunks; ++c) s += part[(size_t)c * N2 * N2 + t];
        dJ[t] += s;
    }
}

// dC partials for spin blockIdx.x, walker chunk blockIdx.y: acc[k][x] += w AinvT[col(k)][x]
template <typename real>
__global__ void __launch_bounds__(256)
k_grad_C(int W, int M, int na, int nb, const uint16_t *__restrict__ occ_list, const real *__restrict__ AinvT,
         const double *__restrict__ wgt, double *__restrict__ part) {
    const int s = blockIdx.x, n = s ? nb : na, ne = na + nb;
    extern __shared__ double acc[];   // [M][n]
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int t = tid; t < M * n; t += nt) acc[t] = 0.0;
    __syncthreads();
    const size_t astride = (size_t)na * na + (size_t)nb * nb;
    const size_t aoff = s ? (size_t)na * na : 0;
    const int w0 = blockIdx.y * kChunkC, w1 = min(W, w0 + kChunkC);
    for (int w = w0; w < w1; ++w) {
        const double c = wgt[w];
        const uint16_t *occ = occ_list + (size_t)w * ne + (s ? na : 0);
        const real *A = AinvT + (size_t)w * astride + aoff;
        for (int t = tid; t < n * n; t += nt) {
            const int col = t / n, x = t - col * n;
            acc[(size_t)occ[col] * n + x] += c * (double)A[t];
        }
    }
    __syncthreads();
    double *dst = part + ((size_t)blockIdx.y * 2 + s) * (size_t)M * (na > nb ? na : nb);
    for (int t = tid; t < M * n; t += nt) dst[t] = acc[t];
}

__global__ void k_reduce_C(int M, int na, int nb, int n_chunks, const double *__restrict__ part,
                           double *__restrict__ dCa, double *__restrict__ dCb) {
    const int nmax = na > nb ? na : nb;
    const int tot = M * na + M * nb;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += gridDim.x * blockDim.x) {
        const int s = t >= M * na;
        const int u = s ? t - M * na : t;
        double sum = 0.0;
        for (int c = 0; c < n_chunks; ++c) sum += part[((size_t)c * 2 + s) * (size_t)M * nmax + u];
        (s ? dCb : dCa)[u] += sum;
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

vmc_status launch_grad(vmc_ctx *ctx, const vmc_walkers *Wk, const double *w, double *dJ, double *dCa,
                       double *dCb) {
    const int W = Wk->W, M = Wk->M, na = Wk->n_alpha, nb = Wk->n_beta, N2 = 2 * M;
    const int T = (N2 + 31) / 32, ntile = T * (T + 1) / 2;
    const int cj = (W + kChunkJ - 1) / kChunkJ, cc = (W + kChunkC - 1) / kChunkC;
    const int nmax = na > nb ? na : nb;
    const size_t bytes_J = sizeof(double) * (size_t)cj * N2 * N2;
    const size_t bytes_C = sizeof(double) * (size_t)cc * 2 * M * nmax;
    vmc_status st = ensure_workspace(ctx, bytes_J > bytes_C ? bytes_J : bytes_C);
    if (st) return st;
    double *part = (double *)ctx->ws;
    if (dJ) {
        k_grad_J<<<dim3(ntile, cj), 256, 0, ctx->stream>>>(W, M, Wk->occ_bits, w, part);
        k_reduce_J<<<(N2 * N2 + 255) / 256, 256, 0, ctx->stream>>>(M, cj, part, dJ);
        ctx->launches += 2;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_check(ctx, e, "k_grad_J");
    }
    if (dCa && dCb) {
        const size_t smem = sizeof(double) * (size_t)M * nmax;
        cudaError_t e;
        if (Wk->precision == VMC_FP64) {
            e = cudaFuncSetAttribute(k_grad_C<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess)
                k_grad_C<double><<<dim3(2, cc), 256, smem, ctx->stream>>>(W, M, na, nb, Wk->occ_list,
                                                                          (const double *)Wk->AinvT, w, part);
        } else {
            e = cudaFuncSetAttribute(k_grad_C<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess)
                k_grad_C<float><<<dim3(2, cc), 256, smem, ctx->stream>>>(W, M, na, nb, Wk->occ_list,
                                                                         (const float *)Wk->AinvT, w, part);
        }
        if (e == cudaSuccess) {
            const int tot = M * na + M * nb;
            k_reduce_C<<<(tot + 255) / 256, 256, 0, ctx->stream>>>(M, na, nb, cc, part, dCa, dCb);
        }
        ctx->launches += 2;
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_check(ctx, e, "k_grad_C");
    }
    return VMC_OK;
}

vmc_status launch_amsgrad(vmc_ctx *ctx, double *p, const double *g, double *m, double *n, size_t np,
                          double alpha, double b1, double b2) {
    if (np == 0) return VMC_OK;
    const int blocks = (int)((np + 255) / 256 < 152 * 8 ? (np + 255) / 256 : 152 * 8);
    k_amsgrad<<<blocks, 256, 0, ctx->stream>>>(p, g, m, n, np, alpha, b1, b2);
    ctx->launches += 1;
    return cuda_check(ctx, cudaGetLastError(), "k_amsgrad");
}

vmc_status launch_walker_reduce(vmc_ctx *ctx, int W, const double *t, const double *e, double *out) {
    k_walker_reduce<<<1, 1024, 0, ctx->stream>>>(W, t, e, out);
    ctx->launches += 1;
    return cuda_check(ctx, cudaGetLastError(), "k_walker_reduce");
}
