// Correlator product (Sec. III.A): psi(n) = prod_l c_l[n_l] x pair Jastrow x Slater determinants.
//
// Correlator l covers a few spatial sites; the Fock state of a site is n_alpha + 2 n_beta and the
// first listed site is the least significant base-4 digit of the coefficient index.  This file
// holds the structure object (per-site lists of the correlators covering each site, so a move's
// ratio only visits the correlators that touch its changed orbitals, Sec. III.B), the walker state
// (one index per correlator), its contribution to ln|psi|, and the gradient ratio
// d ln psi / d c_l[k] = 1/c_l[k] summed over walkers in exact 64-bit fixed point.
// The ratio itself is evaluated inside the local-energy, CTMC and move-set kernels (eloc.cu).
#include <math.h>

#include <vector>

#include "common.cuh"

namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Coefficient index of correlator l for walker w from its occupation bit strings.
__device__ __forceinline__ int cps_index(const CpsView &C, const uint32_t *bits_w, int M, int nw, int l) {
    int idx = 0, mult = 1;
    for (int e = C.corr_off[l]; e < C.corr_off[l + 1]; ++e, mult *= 4) {
        const int k = C.corr_sites[e];
        const int na = (bits_w[k >> 5] >> (k & 31)) & 1, nb = (bits_w[nw + (k >> 5)] >> (k & 31)) & 1;
        idx += (na + 2 * nb) * mult;
    }
    (void)M;
    return idx;
}

__global__ void k_cps_state(CpsView C, int W, int M, const uint32_t *__restrict__ bits, uint16_t *__restrict__ state) {
    const int nw = (M + 31) / 32;
    const int64_t tot = (int64_t)W * C.n_corr;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
        const int w = (int)(t / C.n_corr), l = (int)(t % C.n_corr);
        state[t] = (uint16_t)cps_index(C, bits + (size_t)w * 2 * nw, M, nw, l);
    }
}

// out[w] += sum_l ln|c_l[n_l]| from the walker's occupied lists (no walker table), one CTA per
// walker, summed in a fixed order.
__global__ void __launch_bounds__(128) k_cps_log_psi(CpsView C, int M, int na, int nb,
                                                     const uint16_t *__restrict__ occ, double *__restrict__ out) {
    __shared__ unsigned char s_n[2 * VMC_MAX_M];
    __shared__ double red[4];
    const int w = blockIdx.x, ne = na + nb;
    for (int p = threadIdx.x; p < 2 * M; p += blockDim.x) s_n[p] = 0;
    __syncthreads();
    for (int c = threadIdx.x; c < ne; c += blockDim.x) s_n[(c < na ? 0 : M) + occ[(size_t)w * ne + c]] = 1;
    __syncthreads();
    double acc = 0.0;
    for (int l = threadIdx.x; l < C.n_corr; l += blockDim.x) {
        int idx = 0, mult = 1;
        for (int e = C.corr_off[l]; e < C.corr_off[l + 1]; ++e, mult *= 4) {
            const int k = C.corr_sites[e];
            idx += (s_n[k] + 2 * s_n[M + k]) * mult;
        }
        acc += log(fabs(C.values[C.val_off[l] + idx]));
    }
    acc = warp_sum_f64(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) out[w] += (red[0] + red[1]) + (red[2] + red[3]);
}

// Weights of walker w: mode 0 -> (t[w]); mode 1 -> (t[w], t[w] e[w]) as in the other gradient blocks.
__device__ __forceinline__ double cps_weight(int o, const double *t, const double *e, int w) {
    return o == 0 ? t[w] : t[w] * e[w];
}

// Largest |1/c| over the coefficients the walkers select (positive doubles order like their bits).
__global__ void k_cps_invmax(CpsView C, int W, const uint16_t *__restrict__ state,
                             unsigned long long *__restrict__ inv_max) {
    double m = 0.0;
    const int64_t tot = (int64_t)W * C.n_corr;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
        const int l = (int)(t % C.n_corr);
        if (state[t] >= C.val_off[l + 1] - C.val_off[l]) continue;   // inconsistent state: never read
        m = fmax(m, 1.0 / fabs(C.values[C.val_off[l] + state[t]]));
    }
#pragma unroll
    for (int k = 16; k >= 1; k >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, k));
    if ((threadIdx.x & 31) == 0) atomicMax(inv_max, (unsigned long long)__double_as_longlong(m));
}

// Fixed-point scale per output: 2^s with s = 61 - ilogb(sum_w |weight_w| x max |1/c|), so that no
// partial sum of rounded terms leaves 63 bits.  One CTA, fixed summation order.
__global__ void __launch_bounds__(1024) k_cps_scale(int W, const double *__restrict__ t, const double *__restrict__ e,
                                                    int n_out, const unsigned long long *__restrict__ inv_max,
                                                    int *__restrict__ sexp) {
    __shared__ double r[2][32];
    double a0 = 0.0, a1 = 0.0;
    for (int w = threadIdx.x; w < W; w += blockDim.x) {
        a0 += fabs(cps_weight(0, t, e, w));
        if (n_out > 1) a1 += fabs(cps_weight(1, t, e, w));
    }
    a0 = warp_sum_f64(a0);
    a1 = warp_sum_f64(a1);
    if ((threadIdx.x & 31) == 0) { r[0][threadIdx.x >> 5] = a0; r[1][threadIdx.x >> 5] = a1; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double A0 = 0.0, A1 = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { A0 += r[0][k]; A1 += r[1][k]; }
        const double B = __longlong_as_double((long long)*inv_max);
        sexp[0] = A0 * B > 0.0 ? 61 - ilogb(A0 * B) : 0;
        sexp[1] = A1 * B > 0.0 ? 61 - ilogb(A1 * B) : 0;
    }
}

// acc_o[off_l + n_l] += round(weight_o(w) / c_l[n_l] * 2^s_o): exact, order-independent integer sums.
__global__ void k_cps_grad(CpsView C, int W, const uint16_t *__restrict__ state, const double *__restrict__ t,
                           const double *__restrict__ e, int n_out, const int *__restrict__ sexp,
                           unsigned long long *__restrict__ acc, int64_t n_values) {
    const int64_t tot = (int64_t)W * C.n_corr;
    const int s0 = sexp[0], s1 = sexp[1];
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < tot; x += (int64_t)gridDim.x * blockDim.x) {
        const int w = (int)(x / C.n_corr), l = (int)(x % C.n_corr);
        if (state[x] >= C.val_off[l + 1] - C.val_off[l]) continue;   // inconsistent state: never read
        const int64_t k = C.val_off[l] + state[x];
        const double inv = 1.0 / C.values[k];
        const long long q0 = __double2ll_rn(scalbn(cps_weight(0, t, e, w) * inv, s0));
        atomicAdd(acc + k, (unsigned long long)q0);
        if (n_out > 1) {
            const long long q1 = __double2ll_rn(scalbn(cps_weight(1, t, e, w) * inv, s1));
            atomicAdd(acc + n_values + k, (unsigned long long)q1);
        }
    }
}

__global__ void k_cps_finish(int64_t n_values, int n_out, const unsigned long long *__restrict__ acc,
                             const int *__restrict__ sexp, double *__restrict__ out0, double *__restrict__ out1) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n_values; k += (int64_t)gridDim.x * blockDim.x) {
        out0[k] += scalbn((double)(long long)acc[k], -sexp[0]);
        if (n_out > 1) out1[k] += scalbn((double)(long long)acc[n_values + k], -sexp[1]);
    }
}

__global__ void k_cps_convert(int64_t n, const double *__restrict__ v, float *__restrict__ v32) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        v32[k] = (float)v[k];
}

int grid_for(int64_t n) {
    const int64_t b = (n + 255) / 256;
    return (int)(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}

}  // namespace

CpsView cps_view(const vmc_params *P) {
    CpsView v{};
    if (P && P->cps) {
        v = P->cps->view;
        v.values = P->cps_values;
    }
    return v;
}

vmc_status check_cps(vmc_ctx *ctx, const vmc_params *P, const vmc_walkers *Wk) {
    if (!P || !P->cps) return VMC_OK;
    if (!P->cps_values) return set_err(ctx, VMC_ERR_ARG, "correlator product without coefficients");
    if (P->cps->M != Wk->M) return set_err(ctx, VMC_ERR_ARG, "correlator product and walkers disagree on M");
    if (!Wk->cps_state) return set_err(ctx, VMC_ERR_ARG, "correlator product needs walkers.cps_state");
    return VMC_OK;
}

vmc_status launch_cps_state(vmc_ctx *ctx, const vmc_params *P, vmc_walkers *Wk) {
    const CpsView C = cps_view(P);
    if (!C.n_corr) return VMC_OK;
    k_cps_state<<<grid_for((int64_t)Wk->W * C.n_corr), 256, 0, ctx->stream>>>(C, Wk->W, Wk->M, Wk->occ_bits,
                                                                              Wk->cps_state);
    const int64_t nv = P->cps->n_values;
    k_cps_convert<<<grid_for(nv), 256, 0, ctx->stream>>>(nv, C.values, (float *)C.values32);
    ctx->launches += 2;
    return cuda_check(ctx, cudaGetLastError(), "k_cps_state");
}

vmc_status launch_cps_log_psi(vmc_ctx *ctx, const vmc_params *P, const vmc_walkers *Wk, double *out) {
    const CpsView C = cps_view(P);
    if (!C.n_corr) return VMC_OK;
    k_cps_log_psi<<<Wk->W, 128, 0, ctx->stream>>>(C, Wk->M, Wk->n_alpha, Wk->n_beta, Wk->occ_list, out);
    ctx->launches += 1;
    return cuda_check(ctx, cudaGetLastError(), "k_cps_log_psi");
}

static vmc_status cps_grad(vmc_ctx *ctx, const vmc_walkers *Wk, const vmc_params *P, const double *t, const double *e,
                           int n_out, double *out0, double *out1) {
    const CpsView C = cps_view(P);
    const int64_t nv = P->cps->n_values;
    const size_t bytes = 256 + sizeof(unsigned long long) * (size_t)n_out * nv;
    vmc_status st = ensure_workspace(ctx, bytes);
    if (st) return st;
    unsigned long long *inv_max = (unsigned long long *)ctx->ws;
    int *sexp = (int *)((char *)ctx->ws + 64);
    unsigned long long *acc = (unsigned long long *)((char *)ctx->ws + 256);
    cudaError_t err = cudaMemsetAsync(ctx->ws, 0, bytes, ctx->stream);
    if (err != cudaSuccess) return cuda_check(ctx, err, "cps gradient workspace");
    const int64_t tot = (int64_t)Wk->W * C.n_corr;
    k_cps_invmax<<<grid_for(tot), 256, 0, ctx->stream>>>(C, Wk->W, Wk->cps_state, inv_max);
    k_cps_scale<<<1, 1024, 0, ctx->stream>>>(Wk->W, t, e, n_out, inv_max, sexp);
    k_cps_grad<<<grid_for(tot), 256, 0, ctx->stream>>>(C, Wk->W, Wk->cps_state, t, e, n_out, sexp, acc, nv);
    k_cps_finish<<<grid_for(nv), 256, 0, ctx->stream>>>(nv, n_out, acc, sexp, out0, out1);
    ctx->launches += 4;
    return cuda_check(ctx, cudaGetLastError(), "k_cps_grad");
}

extern "C" {

vmc_status vmc_cps_create(vmc_ctx *ctx, int M, int n_corr, const int32_t *h_off, const int32_t *h_sites,
                          vmc_cps **out) {
    if (!ctx || !out) return ctx ? set_err(ctx, VMC_ERR_ARG, "null argument") : VMC_ERR_ARG;
    *out = nullptr;
    if (!h_off || !h_sites) return set_err(ctx, VMC_ERR_ARG, "null correlator structure");
    if (M < 1 || M > VMC_MAX_M) return set_err(ctx, VMC_ERR_ARG, "M must be in [1, 256]");
    if (n_corr < 1 || n_corr > 65534) return set_err(ctx, VMC_ERR_ARG, "n_corr must be in [1, 65534]");
    if (h_off[0] != 0) return set_err(ctx, VMC_ERR_ARG, "h_off[0] must be 0");
    std::vector<int32_t> val_off(n_corr + 1, 0);
    std::vector<std::vector<uint32_t>> per_site(M);
    for (int l = 0; l < n_corr; ++l) {
        const int k = h_off[l + 1] - h_off[l];
        if (k < 1 || k > VMC_CPS_MAX_SITES) return set_err(ctx, VMC_ERR_ARG, "a correlator must cover 1 to 8 sites");
        for (int t = 0; t < k; ++t) {
            const int site = h_sites[h_off[l] + t];
            if (site < 0 || site >= M) return set_err(ctx, VMC_ERR_ARG, "correlator site outside [0, M)");
            for (int u = 0; u < t; ++u)
                if (h_sites[h_off[l] + u] == site) return set_err(ctx, VMC_ERR_ARG, "repeated site in a correlator");
            per_site[site].push_back(((uint32_t)l << 16) | (1u << (2 * t)));
        }
        if ((int64_t)val_off[l] + ((int64_t)1 << (2 * k)) > 0x7FFFFFFF)
            return set_err(ctx, VMC_ERR_ARG, "more than 2^31 - 1 coefficients");
        val_off[l + 1] = val_off[l] + (1 << (2 * k));
    }
    std::vector<int32_t> site_off(M + 1, 0);
    std::vector<uint32_t> site_ent;
    for (int k = 0; k < M; ++k) {
        if ((int)per_site[k].size() > VMC_CPS_MAX_PER_SITE)
            return set_err(ctx, VMC_ERR_ARG, "more than 16 correlators cover one site");
        site_ent.insert(site_ent.end(), per_site[k].begin(), per_site[k].end());   // l ascending
        site_off[k + 1] = (int32_t)site_ent.size();
    }
    const size_t nnz = (size_t)h_off[n_corr];
    vmc_cps *c = new vmc_cps();
    c->M = M;
    c->n_corr = n_corr;
    c->n_values = val_off[n_corr];
    c->nnz = (int)nnz;
    size_t o_off = 0, o_sites = align256(o_off + sizeof(int32_t) * (n_corr + 1));
    size_t o_val = align256(o_sites + sizeof(int32_t) * nnz);
    size_t o_soff = align256(o_val + sizeof(int32_t) * (n_corr + 1));
    size_t o_ent = align256(o_soff + sizeof(int32_t) * (M + 1));
    size_t o_v32 = align256(o_ent + sizeof(uint32_t) * (site_ent.size() + 1));
    size_t total = align256(o_v32 + sizeof(float) * (size_t)c->n_values);
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e == cudaSuccess) e = cudaMalloc(&c->dev, total);
    char *b = (char *)c->dev;
    if (e == cudaSuccess) e = cudaMemcpy(b + o_off, h_off, sizeof(int32_t) * (n_corr + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b + o_sites, h_sites, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b + o_val, val_off.data(), sizeof(int32_t) * (n_corr + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b + o_soff, site_off.data(), sizeof(int32_t) * (M + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !site_ent.empty())
        e = cudaMemcpy(b + o_ent, site_ent.data(), sizeof(uint32_t) * site_ent.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        vmc_cps_destroy(c);
        return cuda_check(ctx, e, "correlator structure upload");
    }
    CpsView &v = c->view;
    v.n_corr = n_corr;
    v.M = M;
    v.nnz = (int)nnz;
    v.corr_off = (const int32_t *)(b + o_off);
    v.corr_sites = (const int32_t *)(b + o_sites);
    v.val_off = (const int32_t *)(b + o_val);
    v.values32 = (const float *)(b + o_v32);
    v.site_off = (const int32_t *)(b + o_soff);
    v.site_ent = (const uint32_t *)(b + o_ent);
    v.values = nullptr;
    *out = c;
    return VMC_OK;
}

vmc_status vmc_cps_destroy(vmc_cps *c) {
    if (!c) return VMC_OK;
    if (c->dev) cudaFree(c->dev);
    delete c;
    return VMC_OK;
}

vmc_status vmc_cps_info(const vmc_cps *c, int *n_corr, int64_t *n_values) {
    if (!c) return VMC_ERR_ARG;
    if (n_corr) *n_corr = c->n_corr;
    if (n_values) *n_values = c->n_values;
    return VMC_OK;
}

vmc_status vmc_grad_logpsi_cps(vmc_ctx *ctx, const vmc_walkers *Wk, const vmc_params *P, const double *w, double *dc) {
    if (!ctx) return VMC_ERR_ARG;
    if (!Wk || !P || !P->cps || !w || !dc) return set_err(ctx, VMC_ERR_ARG, "null argument");
    if (Wk->W < 1) return set_err(ctx, VMC_ERR_ARG, "W must be >= 1");
    vmc_status st = check_cps(ctx, P, Wk);
    if (st) return st;
    return cps_grad(ctx, Wk, P, w, nullptr, 1, dc, nullptr);
}

vmc_status vmc_accumulate_gradient_cps(vmc_ctx *ctx, const vmc_walkers *Wk, const vmc_params *P, const double *t,
                                       const double *e, double *aO, double *aEO) {
    if (!ctx) return VMC_ERR_ARG;
    if (!Wk || !P || !P->cps || !t || !e || !aO || !aEO) return set_err(ctx, VMC_ERR_ARG, "null argument");
    if (Wk->W < 1) return set_err(ctx, VMC_ERR_ARG, "W must be >= 1");
    vmc_status st = check_cps(ctx, P, Wk);
    if (st) return st;
    return cps_grad(ctx, Wk, P, t, e, 2, aO, aEO);
}

}  // extern "C"
