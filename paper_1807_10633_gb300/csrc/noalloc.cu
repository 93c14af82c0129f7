// vmc_grad_logpsi_noalloc: the vector-Jacobian product of ln psi without any allocation.
//
// Some callers cannot allocate device memory at all: services that give a framework's pooling
// allocator sole control of the device (a cudaMalloc behind its back can fail or fragment its
// pool), fixed-footprint deployments that reserve every byte up front, and host loops that must
// not stall (cudaMalloc and cudaFree may synchronise with the device).  This entry
// point needs neither cudaMalloc nor a context: its scratch space (fixed-point weights and
// per-chunk partial sums) is a file-scope device array of VMC_NOALLOC_SCRATCH_BYTES that every
// GPU loading the library holds until the process exits.  The caller still passes the walker
// arrays, the weights and the outputs.
//
// Set-up: the first call on a device (with that device current) looks up the array's device
// address with cudaGetSymbolAddress and caches it; make that first call before any stream
// capture.  All calls share the one array, so calls that overlap on the GPU race; each call
// writes every scratch location it reads before reading it.
#include <math.h>
#include <mutex>

#include "common.cuh"

#define VMC_NOALLOC_SCRATCH_BYTES (16u << 20)
#define VMC_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) unsigned char g_noalloc_scratch[VMC_NOALLOC_SCRATCH_BYTES];

namespace {

std::mutex g_setup_mutex;
void *g_scratch_ptr[VMC_NOALLOC_MAX_DEVICES] = {nullptr};

constexpr int kRows = 16;   // orbital rows per CTA for the orbital block

__device__ __forceinline__ uint32_t nb_window_bits(const uint32_t *bits_w, int M, int nw, int p0, int lane) {
    const int p = p0 + lane;
    int bit = 0;
    if (p < 2 * M) {
        const int s = p >= M, k = p - s * M;
        bit = (bits_w[s * nw + (k >> 5)] >> (k & 31)) & 1;
    }
    return __ballot_sync(0xffffffffu, bit);
}

// Fixed-point weights cq = round(w 2^s), s from sum |w| (no partial sum can overflow 63 bits).
__global__ void __launch_bounds__(1024)
nb_weight_prep(int W, const double *__restrict__ wgt, long long *__restrict__ cq, int *__restrict__ sexp) {
    __shared__ double r[32];
    __shared__ int s_exp;
    double a = 0.0;
    for (int w = threadIdx.x; w < W; w += blockDim.x) a += fabs(wgt[w]);
    a = warp_sum_f64(a);
    if ((threadIdx.x & 31) == 0) r[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double A = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) A += r[k];
        s_exp = A > 0.0 ? 61 - ilogb(A) : 0;
        *sexp = s_exp;
    }
    __syncthreads();
    for (int w = threadIdx.x; w < W; w += blockDim.x) cq[w] = __double2ll_rn(scalbn(wgt[w], s_exp));
}

// Jastrow block partials, tile (P,Q) P<=Q of 32x32 spin orbitals, walker chunk blockIdx.y.
__global__ void __launch_bounds__(256)
nb_grad_J(int W, int M, int chunk, const uint32_t *__restrict__ bits, const long long *__restrict__ cq,
          long long *__restrict__ part) {
    const int N2 = 2 * M, nw = (M + 31) / 32, T = (N2 + 31) / 32;
    int t = blockIdx.x, P = 0;
    while (t >= T - P) { t -= T - P; ++P; }
    const int Q = P + t;
    const int tid = threadIdx.x, lane = tid & 31;
    const int pl = tid >> 3, ql0 = (tid & 7) * 4;
    long long acc[4] = {0, 0, 0, 0};
    const int w0 = blockIdx.y * chunk, w1 = min(W, w0 + chunk);
    for (int w = w0; w < w1; ++w) {
        const uint32_t *bw = bits + (size_t)w * 2 * nw;
        const uint32_t bp = nb_window_bits(bw, M, nw, P * 32, lane);
        const uint32_t bq = nb_window_bits(bw, M, nw, Q * 32, lane);
        if ((bp >> pl) & 1u) {
            const long long c = cq[w];
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if ((bq >> (ql0 + k)) & 1u) acc[k] += c;
        }
    }
    long long *dst = part + (size_t)blockIdx.y * N2 * N2;
    const int p = P * 32 + pl;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int q = Q * 32 + ql0 + k;
        if (p < N2 && q < N2 && p <= q) dst[(size_t)p * N2 + q] = acc[k];
    }
}

__global__ void nb_reduce_J(int M, int n_chunks, const long long *__restrict__ part, const int *__restrict__ sexp,
                            double *__restrict__ dJ) {
    const int N2 = 2 * M;
    const int e0 = *sexp;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < N2 * N2; t += gridDim.x * blockDim.x) {
        if (t / N2 > t % N2) continue;
        long long s = 0;
        for (int c = 0; c < n_chunks; ++c) s += part[(size_t)c * N2 * N2 + t];
        dJ[t] += scalbn((double)s, -e0);
    }
}

// Orbital block partials: CTA = (spin, block of kRows orbital rows) x walker chunk.
template <typename real, typename acc_t>
__global__ void __launch_bounds__(128)
nb_grad_C(int W, int M, int na, int nb, int chunk, const uint16_t *__restrict__ pos,
          const real *__restrict__ AinvT, const double *__restrict__ wgt, double *__restrict__ part) {
    const int nrb = (M + kRows - 1) / kRows;
    const int s = blockIdx.x / nrb, rb = blockIdx.x - s * nrb;
    const int n = s ? nb : na, x = threadIdx.x;
    const int k0 = rb * kRows;
    acc_t acc[kRows];
#pragma unroll
    for (int r = 0; r < kRows; ++r) acc[r] = 0;
    const size_t astride = (size_t)na * na + (size_t)nb * nb;
    const size_t aoff = s ? (size_t)na * na : 0;
    const int w0 = blockIdx.y * chunk, w1 = min(W, w0 + chunk);
    const bool xin = x < n;
    for (int w = w0; w < w1; ++w) {
        const acc_t c = (acc_t)wgt[w];
        const uint16_t *pw = pos + (size_t)w * 2 * M + (size_t)s * M + k0;
        const real *A = AinvT + (size_t)w * astride + aoff;
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            if (k0 + r >= M) break;
            const uint16_t pc = pw[r];
            if (!(pc & 0x8000) && xin) acc[r] += c * (acc_t)A[(size_t)pc * n + x];
        }
    }
    if (!xin) return;
    double *dst = part + ((size_t)blockIdx.y * 2 + s) * (size_t)M * (na > nb ? na : nb);
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        if (k0 + r >= M) break;
        dst[(size_t)(k0 + r) * n + x] = (double)acc[r];
    }
}

__global__ void nb_reduce_C(int M, int na, int nb, int n_chunks, const double *__restrict__ part,
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

// Device address of the scratch array on the current device (looked up once per device).
cudaError_t scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= VMC_NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" vmc_status vmc_grad_logpsi_noalloc(const vmc_walkers *Wk, const double *w, double *dJ, double *dCa,
                                              double *dCb, void *cuda_stream) {
    if (!Wk || !w || !dJ || !dCa || !dCb) return VMC_ERR_ARG;
    if (Wk->W < 1 || Wk->M < 1 || Wk->M > VMC_MAX_M || Wk->n_alpha < 0 || Wk->n_beta < 0 ||
        Wk->n_alpha > Wk->M || Wk->n_beta > Wk->M || !Wk->occ_bits || !Wk->pos || !Wk->AinvT)
        return VMC_ERR_ARG;
    if (Wk->precision != VMC_FP64 && Wk->precision != VMC_MIXED) return VMC_ERR_ARG;
    const int W = Wk->W, M = Wk->M, na = Wk->n_alpha, nb = Wk->n_beta, N2 = 2 * M;
    const int nmax = na > nb ? na : nb;
    if (nmax < 1 || nmax > 128) return VMC_ERR_ARG;
    // scratch layout: [exponent | pad to 256] [cq: W int64] [partials]
    const size_t head = 256 + (((size_t)W * 8 + 255) & ~(size_t)255);
    const size_t jchunk_bytes = (size_t)N2 * N2 * 8, cchunk_bytes = (size_t)2 * M * nmax * 8;
    if (head + jchunk_bytes > VMC_NOALLOC_SCRATCH_BYTES || head + cchunk_bytes > VMC_NOALLOC_SCRATCH_BYTES)
        return VMC_ERR_ARG;   // beyond the fixed scratch size
    const size_t room = VMC_NOALLOC_SCRATCH_BYTES - head;
    int nj = (int)(room / jchunk_bytes), nc = (int)(room / cchunk_bytes);
    nj = nj < (W + 1023) / 1024 ? nj : (W + 1023) / 1024;
    nc = nc < (W + 255) / 256 ? nc : (W + 255) / 256;
    if (nj < 1) nj = 1;
    if (nc < 1) nc = 1;
    const int cj = (W + nj - 1) / nj, cc = (W + nc - 1) / nc;
    nj = (W + cj - 1) / cj;
    nc = (W + cc - 1) / cc;
    void *base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) return VMC_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int *sexp = (int *)base;
    long long *cq = (long long *)((char *)base + 256);
    void *part = (char *)base + head;
    const int T = (N2 + 31) / 32, ntile = T * (T + 1) / 2;
    nb_weight_prep<<<1, 1024, 0, st>>>(W, w, cq, sexp);
    nb_grad_J<<<dim3(ntile, nj), 256, 0, st>>>(W, M, cj, Wk->occ_bits, cq, (long long *)part);
    nb_reduce_J<<<(N2 * N2 + 255) / 256, 256, 0, st>>>(M, nj, (const long long *)part, sexp, dJ);
    const int nrb = (M + kRows - 1) / kRows, threads = ((nmax + 31) / 32) * 32;
    if (Wk->precision == VMC_FP64)
        nb_grad_C<double, double><<<dim3(2 * nrb, nc), threads, 0, st>>>(W, M, na, nb, cc, Wk->pos,
                                                                         (const double *)Wk->AinvT, w, (double *)part);
    else
        nb_grad_C<float, float><<<dim3(2 * nrb, nc), threads, 0, st>>>(W, M, na, nb, cc, Wk->pos,
                                                                       (const float *)Wk->AinvT, w, (double *)part);
    const int tot = M * na + M * nb;
    nb_reduce_C<<<(tot + 255) / 256, 256, 0, st>>>(M, na, nb, nc, (const double *)part, dCa, dCb);
    e = cudaGetLastError();
    return e == cudaSuccess ? VMC_OK : VMC_ERR_CUDA;
}
