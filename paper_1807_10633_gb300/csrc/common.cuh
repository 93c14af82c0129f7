// Internal definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "vmc.h"

typedef unsigned __int128 u128;

#define VMC_MAX_M 256
#define VMC_WARPS 8
#define VMC_THREADS (VMC_WARPS * 32)

// Device status word bits (latched, cleared by vmc_sync).
#define VMC_DEV_SINGULAR 1u
#define VMC_DEV_OVERFLOW 2u
#define VMC_DEV_NOMOVE 4u
#define VMC_DEV_INCONSISTENT 8u
#define VMC_DEV_TIMEOUT 16u

struct vmc_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    unsigned int *d_status = nullptr;
    std::string err;
    void *ws = nullptr;          // scratch for gradient partial sums
    size_t ws_bytes = 0;
    void *rates = nullptr;       // CTMC rate store: per walker, per group, 128-bit sums
    size_t rates_bytes = 0;
    // rate store bookkeeping (vmc_local_energy -> vmc_ctmc_step)
    const void *rates_walkers = nullptr;
    int rates_valid = 0;
    int rates_groups = 0;
    uint64_t launches = 0;
    // batched launches: device descriptor table (re-uploaded only when the batch changes)
    void *batch_desc = nullptr;
    size_t batch_desc_bytes = 0;
    std::string batch_host;
    int *d_queue = nullptr;
    std::string rates_batch;       // walker tables the batched rate store belongs to
    int eloc_threads = 256;        // threads per local-energy CTA (set by the autotuner)
    int g_tensor_cores = 1;        // refresh: G on tcgen05 (1) or CUDA cores (0)
    int refresh_smem = 0;          // refresh: register Gauss-Jordan (0) or shared-memory LU/GJ (1)
    int mixed_gj32 = 0;            // mixed refresh: FP64 LU of C_occ (0) or FP32 register Gauss-Jordan (1)
    int grad_j_tc = 1;             // Jastrow walker sums: tcgen05 digit products (1) or integer pipe (0)
};

// Plain-pointer view of the device lists, passed to kernels by value.
struct ListsView {
    int M;
    int band;      // largest |p - q| with a non-empty double list (pair candidates of a row)
    int cpr;       // warp chunks (32 candidates) per alpha row
    int rpg;       // beta rows per group (their candidates are the band's same-spin q only)
    int cpr_b;     // warp chunks per beta row when rpg == 1
    int n_groups;  // singles blocks of 32 spin orbitals + M * cpr alpha-row chunks + beta groups
    int64_t ns, nds, ndo;
    int64_t ns_pad;          // ns rounded up to a multiple of 4: row stride of the Fock tables and of F
    // singles, CSR over spatial i; records {a, w_alpha, w_beta, 0}: 16 B (mixed) or 32 B (FP64,
    // the first 8 bytes hold a)
    const uint32_t *s_off, *s_len, *s_owner;
    const uint16_t *s_a;
    const float4 *s_rec32;
    const double4_32a *s_rec64;
    // same-spin doubles, CSR over tri(p<q); records: mixed {ab, v, w_alpha, w_beta},
    // FP64 {ab, v, w_alpha, w_beta} with ab in the first 8 bytes
    const uint32_t *ds_off, *ds_len, *ds_ab, *ds_owner;
    const float4 *ds_rec32;
    const double4_32a *ds_rec64;
    // opposite-spin doubles, CSR over p*M+q; records {ab, v, w, 0}
    const uint32_t *do_off, *do_len, *do_ab, *do_owner;
    const float4 *do_rec32;
    const double4_32a *do_rec64;
    // Fock-sum update tables: Tj[k][e] = (ai|kk), Tjk[k][e] = (ai|kk) - (ak|ki), rows of ns_pad
    // (zero padded); FP64 and FP32 copies
    const double *Tj, *Tjk;
    const float *Tjf, *Tjkf;
    // diagonal tables: Jd[p][q] = (pp|qq), Kd[p][q] = (pq|qp); hd[p] = h_pp; h1 full
    const double *Jd, *Kd, *hd, *h1;
    double e_core;
    // work units of the local energy, [n_groups][32] in canonical order: {key naming the unit's own
    // orbitals (a | b << 16, spatial for kinds 0-1, alpha | beta << 16 for kind 2), list base,
    // list length at the current eps_run (0: no unit), kind | spin << 2}
    const uint4 *unit_tab;
};

// Correlator product (Sec. III.A): device view of the structure plus the coefficient table.
#define VMC_CPS_MAX_SITES 8        // sites per correlator: 4^8 coefficients, a 16-bit index
#define VMC_CPS_MAX_PER_SITE 16    // correlators covering one site
struct CpsView {
    int n_corr;                    // 0: no correlator product
    int M, nnz;                    // orbitals; total sites over the correlators (= site_ent entries)
    const int32_t *corr_off;       // [n_corr + 1]: sites of correlator l are corr_sites[corr_off[l] ..)
    const int32_t *corr_sites;
    const int32_t *val_off;        // [n_corr + 1]: coefficients of l at values[val_off[l] ..], 4^k of them
    const int32_t *site_off;       // [M + 1]: correlators covering site k are site_ent[site_off[k] ..)
    const uint32_t *site_ent;      // (l << 16) | 4^t, t = the site's digit position in l; l ascending
    const double *values;          // the coefficients (parameters), FP64, device
    const float *values32;         // FP32 copy made by the last walker (re)initialisation (mixed form)
};

struct vmc_cps {
    int M = 0, n_corr = 0, nnz = 0;
    int64_t n_values = 0;
    void *dev = nullptr;           // one device allocation: offsets, sites, site table, FP32 copy
    CpsView view{};                // values == nullptr (passed with the parameters)
};

struct vmc_lists {
    int M = 0;
    double eps_build = 0.0;
    double eps_run = -1.0;   // eps the effective lengths were computed for
    int64_t near_ties_build = 0;   // near ties of the build eps over every candidate (Sec. II.A)
    int64_t ns = 0, nds = 0, ndo = 0;
    // host copies of the sorted magnitudes (for effective lengths at a given eps_run)
    double *h_s_key = nullptr, *h_ds_key = nullptr, *h_do_key = nullptr;
    uint32_t *h_s_off = nullptr, *h_ds_off = nullptr, *h_do_off = nullptr;
    void *dev = nullptr;     // one device allocation holding every array
    size_t dev_bytes = 0;
    ListsView view{};
    void *cf = nullptr;      // FP32 copy of C_alpha | C_beta (M x 2M floats at most)
    void *cdig = nullptr;    // FP64-form G: BF16 digit table of C and its row exponents
    void *jsym = nullptr;    // symmetric copies of J: FP64 (2M)^2 then FP32 (2M)^2
    const double *jastrow_for = nullptr;   // J pointer the constants were refreshed for
    uint64_t jastrow_epoch = 0;
};

// ------------------------------------------------------------------ small helpers
__host__ __device__ inline int tri_index(int p, int q, int M) {  // p < q
    return p * (2 * M - p - 1) / 2 + (q - p - 1);
}

// J read from the upper triangle only
// Rate store of one system, in 16-byte units: W x n_groups exact rate sums (u128) followed by the
// W x n_groups per-group energy partials (FP64) that the local energy adds in a fixed order.
inline size_t rate_store_units(size_t W, int n_groups) {
    const size_t n = W * (size_t)n_groups;
    return n + (n + 1) / 2;
}

__device__ __forceinline__ double jget(const double *J, int N2, int p, int q) {
    return p <= q ? J[(size_t)p * N2 + q] : J[(size_t)q * N2 + p];
}

// floor(r * 2^64) as an exact 128-bit integer for r >= 0 (r < 2^43 is the caller's job)
__device__ __forceinline__ u128 rate_fixed(double r) {
    const uint64_t bits = (uint64_t)__double_as_longlong(r);
    const int ex = (int)((bits >> 52) & 0x7FF);
    if (ex == 0) return 0;                       // zero and subnormals (< 2^-1022)
    const uint64_t mant = (bits & ((1ull << 52) - 1)) | (1ull << 52);
    const int sh = ex - 1011;                    // r * 2^64 = mant * 2^sh
    if (sh >= 0) return ((u128)mant) << sh;
    if (sh <= -64) return 0;
    return (u128)(mant >> (-sh));
}
__device__ __forceinline__ u128 rate_fixed(float r) {
    const uint32_t bits = __float_as_uint(r);
    const int ex = (int)((bits >> 23) & 0xFF);
    if (ex == 0) return 0;
    const uint64_t mant = (bits & ((1u << 23) - 1)) | (1u << 23);
    const int sh = ex - 86;                      // r = mant 2^(ex-150); r 2^64 = mant 2^(ex-86)
    if (sh >= 0) return ((u128)mant) << sh;
    if (sh <= -64) return 0;
    return (u128)(mant >> (-sh));
}

__device__ __forceinline__ u128 shfl_xor_u128(u128 v, int m) {
    uint64_t lo = (uint64_t)v, hi = (uint64_t)(v >> 64);
    lo = __shfl_xor_sync(0xffffffffu, lo, m);
    hi = __shfl_xor_sync(0xffffffffu, hi, m);
    return ((u128)hi << 64) | lo;
}
__device__ __forceinline__ u128 shfl_up_u128(u128 v, int d) {
    uint64_t lo = (uint64_t)v, hi = (uint64_t)(v >> 64);
    lo = __shfl_up_sync(0xffffffffu, lo, d);
    hi = __shfl_up_sync(0xffffffffu, hi, d);
    return ((u128)hi << 64) | lo;
}
__device__ __forceinline__ u128 shfl_u128(u128 v, int src) {
    uint64_t lo = (uint64_t)v, hi = (uint64_t)(v >> 64);
    lo = __shfl_sync(0xffffffffu, lo, src);
    hi = __shfl_sync(0xffffffffu, hi, src);
    return ((u128)hi << 64) | lo;
}
__device__ __forceinline__ u128 warp_sum_u128(u128 v) {
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) v += shfl_xor_u128(v, m);
    return v;
}
__device__ __forceinline__ u128 warp_incl_scan_u128(u128 v, int lane) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        u128 o = shfl_up_u128(v, d);
        if (lane >= d) v += o;
    }
    return v;
}
__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
    return v;
}

// Philox4x64-10 (Salmon et al., SC'11): ten rounds, two 64x64->128 products per round.
__device__ __forceinline__ uint64_t philox4x64_word0(uint64_t c0, uint64_t c1, uint64_t c2,
                                                     uint64_t c3, uint64_t k0, uint64_t k1) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
        const uint64_t hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
        const uint64_t y0 = hi1 ^ c1 ^ k0, y2 = hi0 ^ c3 ^ k1;
        c0 = y0; c1 = lo1; c2 = y2; c3 = lo0;
        k0 += W0; k1 += W1;
    }
    return c0;
}

// ------------------------------------------------------------------ host-side helpers
vmc_status set_err(vmc_ctx *ctx, vmc_status st, const std::string &msg);
vmc_status cuda_check(vmc_ctx *ctx, cudaError_t e, const char *what);
vmc_status ensure_workspace(vmc_ctx *ctx, size_t bytes);
size_t walker_stride_G(int M, int na, int nb);
size_t walker_stride_A(int na, int nb);

// launchers (defined in the .cu files)
vmc_status launch_refresh_jastrow(vmc_ctx *ctx, vmc_lists *L, const double *J);
vmc_status launch_init_walkers(vmc_ctx *ctx, vmc_lists *L, const vmc_params *P,
                               vmc_walkers *Wk, int full);
struct CpsView;
vmc_status launch_local_energy(vmc_ctx *ctx, const vmc_lists *L, vmc_walkers *Wk, const CpsView &C,
                               double *e_loc, double *t_res, u128 *rates, int n_groups);
vmc_status launch_ctmc_step(vmc_ctx *ctx, const vmc_lists *L, const vmc_params *P,
                            vmc_walkers *Wk, uint64_t seed, const u128 *rates, int n_groups,
                            uint64_t *move_code);
vmc_status launch_screened_moves(vmc_ctx *ctx, const vmc_lists *L, const vmc_walkers *Wk, const CpsView &C,
                                 int w_begin, int n_w, int64_t cap, uint64_t *code, double *ratio, double *contrib,
                                 int64_t *count, int64_t *walked);
vmc_status launch_local_energy_batch(vmc_ctx *ctx, int n, const vmc_batch_item *items);
vmc_status launch_ctmc_step_batch(vmc_ctx *ctx, int n, const vmc_batch_item *items, uint64_t seed);
vmc_status launch_g_umma(vmc_ctx *ctx, const vmc_walkers *Wk, const float *Cf);
size_t g_umma_smem(int M, int na, int nb);
bool g_ozaki_ok(int M, int na, int nb);
size_t g_ozaki_table_bytes(int M);
vmc_status launch_g_ozaki(vmc_ctx *ctx, const vmc_walkers *Wk, const double *Ca, const double *Cb, void *table);
vmc_status launch_grad_J_umma(vmc_ctx *ctx, int W, int M, const uint32_t *bits, const long long *cq, int mode,
                              long long *part, int chunk, int n_chunks);
void grad_j_umma_chunks(int W, int M, int nsm, int *chunk, int *n_chunks);
vmc_status launch_grad(vmc_ctx *ctx, const vmc_walkers *Wk, const double *w, double *dJ,
                       double *dCa, double *dCb);
vmc_status launch_accumulate(vmc_ctx *ctx, const vmc_walkers *Wk, const double *t, const double *e,
                             double *const aO[3], double *const aEO[3], double *sums);
vmc_status launch_amsgrad(vmc_ctx *ctx, double *p, const double *g, double *m, double *n,
                          size_t np, double alpha, double b1, double b2);
vmc_status launch_energy_gradient(vmc_ctx *ctx, size_t n, const double *sums, const double *aO,
                                  const double *aEO, double *g);
vmc_status launch_walker_reduce(vmc_ctx *ctx, int W, const double *t, const double *e,
                                double *out);
vmc_status launch_log_psi(vmc_ctx *ctx, const vmc_walkers *Wk, const vmc_params *P,
                          double *out);
// correlator product (cps.cu)
CpsView cps_view(const vmc_params *P);
vmc_status check_cps(vmc_ctx *ctx, const vmc_params *P, const vmc_walkers *Wk);
vmc_status launch_cps_state(vmc_ctx *ctx, const vmc_params *P, vmc_walkers *Wk);
vmc_status launch_cps_log_psi(vmc_ctx *ctx, const vmc_params *P, const vmc_walkers *Wk, double *out);
