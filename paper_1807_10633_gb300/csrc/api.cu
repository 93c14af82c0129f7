// C-ABI entry points: argument checks, context and workspace management, call ordering.
#include <stdio.h>
#include <string.h>

#include <string>

#include "common.cuh"

vmc_status lists_set_eps(vmc_ctx *ctx, vmc_lists *L, double eps_run);

vmc_status set_err(vmc_ctx *ctx, vmc_status st, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return st;
}

vmc_status cuda_check(vmc_ctx *ctx, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return VMC_OK;
    if (e == cudaErrorMemoryAllocation)
        return set_err(ctx, VMC_ERR_OOM, std::string(what) + ": " + cudaGetErrorString(e));
    return set_err(ctx, VMC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

vmc_status ensure_workspace(vmc_ctx *ctx, size_t bytes) {
    if (bytes <= ctx->ws_bytes) return VMC_OK;
    if (ctx->ws) {
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return cuda_check(ctx, e, "workspace resize");
        cudaFree(ctx->ws);
        ctx->ws = nullptr;
        ctx->ws_bytes = 0;
    }
    cudaError_t e = cudaMalloc(&ctx->ws, bytes);
    if (e != cudaSuccess) return cuda_check(ctx, e, "workspace");
    ctx->ws_bytes = bytes;
    return VMC_OK;
}

static vmc_status ensure_rates(vmc_ctx *ctx, size_t bytes, void **out) {
    static_assert(sizeof(u128) == 16, "u128");
    // the rate store has its own allocation: it must survive the gradient's use of ctx->ws
    if (bytes > ctx->rates_bytes) {
        if (ctx->rates) {
            cudaError_t e = cudaStreamSynchronize(ctx->stream);
            if (e != cudaSuccess) return cuda_check(ctx, e, "rate store resize");
            cudaFree(ctx->rates);
            ctx->rates = nullptr;
            ctx->rates_bytes = 0;
        }
        cudaError_t e = cudaMalloc(&ctx->rates, bytes);
        if (e != cudaSuccess) return cuda_check(ctx, e, "rate store");
        ctx->rates_bytes = bytes;
    }
    *out = ctx->rates;
    return VMC_OK;
}

size_t walker_stride_G(int M, int na, int nb) { return (size_t)(M - na) * na + (size_t)(M - nb) * nb; }
size_t walker_stride_A(int na, int nb) { return (size_t)na * na + (size_t)nb * nb; }

static vmc_status check_walkers(vmc_ctx *ctx, const vmc_walkers *Wk, const vmc_lists *L) {
    if (!Wk) return set_err(ctx, VMC_ERR_ARG, "null walkers");
    if (Wk->W < 1) return set_err(ctx, VMC_ERR_ARG, "W must be >= 1");
    if (Wk->M < 1 || Wk->M > VMC_MAX_M) return set_err(ctx, VMC_ERR_ARG, "M must be in [1, 256]");
    if (Wk->n_alpha < 0 || Wk->n_beta < 0 || Wk->n_alpha > Wk->M || Wk->n_beta > Wk->M)
        return set_err(ctx, VMC_ERR_ARG, "electron counts out of range");
    if (Wk->n_alpha + Wk->n_beta < 1) return set_err(ctx, VMC_ERR_ARG, "no electrons");
    if (Wk->precision != VMC_FP64 && Wk->precision != VMC_MIXED) return set_err(ctx, VMC_ERR_ARG, "bad precision");
    if (!Wk->occ_bits || !Wk->occ_list || !Wk->virt_list || !Wk->pos || !Wk->G || !Wk->AinvT || !Wk->S || !Wk->F ||
        !Wk->e_diag || !Wk->rng_counter)
        return set_err(ctx, VMC_ERR_ARG, "null walker array");
    if (L && L->M != Wk->M) return set_err(ctx, VMC_ERR_ARG, "lists and walkers disagree on M");
    return VMC_OK;
}

extern "C" {

vmc_status vmc_create(vmc_ctx **out, int device, void *stream) {
    if (!out) return VMC_ERR_ARG;
    *out = nullptr;
    vmc_ctx *ctx = new vmc_ctx();
    ctx->device = device;
    ctx->stream = (cudaStream_t)stream;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_status, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_status, 0, sizeof(unsigned int));
    if (e != cudaSuccess) {
        delete ctx;
        return e == cudaErrorMemoryAllocation ? VMC_ERR_OOM : VMC_ERR_CUDA;
    }
    *out = ctx;
    return VMC_OK;
}

vmc_status vmc_destroy(vmc_ctx *ctx) {
    if (!ctx) return VMC_OK;
    cudaStreamSynchronize(ctx->stream);
    if (ctx->d_status) cudaFree(ctx->d_status);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->rates) cudaFree(ctx->rates);
    if (ctx->batch_desc) cudaFree(ctx->batch_desc);
    if (ctx->d_queue) cudaFree(ctx->d_queue);
    delete ctx;
    return VMC_OK;
}

vmc_status vmc_set_stream(vmc_ctx *ctx, void *stream) {
    if (!ctx) return VMC_ERR_ARG;
    ctx->stream = (cudaStream_t)stream;
    return VMC_OK;
}

vmc_status vmc_set_option(vmc_ctx *ctx, int option, int value) {
    if (!ctx) return VMC_ERR_ARG;
    if (option == VMC_OPT_G_TENSOR_CORES) {
        ctx->g_tensor_cores = value ? 1 : 0;
        return VMC_OK;
    }
    if (option == VMC_OPT_ELOC_THREADS) {
        if (value != 128 && value != 256 && value != 384 && value != 512)
            return set_err(ctx, VMC_ERR_ARG, "128, 256, 384 or 512 threads");
        ctx->eloc_threads = value;
        return VMC_OK;
    }
    if (option == VMC_OPT_REFRESH_SMEM) {
        ctx->refresh_smem = value ? 1 : 0;
        return VMC_OK;
    }
    if (option == VMC_OPT_MIXED_REFRESH_GJ32) {
        ctx->mixed_gj32 = value ? 1 : 0;
        return VMC_OK;
    }
    if (option == VMC_OPT_GRAD_J_TENSOR_CORES) {
        ctx->grad_j_tc = value ? 1 : 0;
        return VMC_OK;
    }
    return set_err(ctx, VMC_ERR_ARG, "unknown option");
}

const char *vmc_last_error(const vmc_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

uint64_t vmc_launch_count(const vmc_ctx *ctx) { return ctx ? ctx->launches : 0; }

vmc_status vmc_sync(vmc_ctx *ctx) {
    if (!ctx) return VMC_ERR_ARG;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_check(ctx, e, "vmc_sync");
    unsigned int st = 0;
    e = cudaMemcpy(&st, ctx->d_status, sizeof(st), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(ctx->d_status, 0, sizeof(unsigned int));
    if (e != cudaSuccess) return cuda_check(ctx, e, "vmc_sync status");
    if (st & VMC_DEV_SINGULAR) return set_err(ctx, VMC_ERR_SINGULAR, "singular C_occ block");
    if (st & VMC_DEV_OVERFLOW) return set_err(ctx, VMC_ERR_OVERFLOW, "CTMC rate reached 2^43");
    if (st & VMC_DEV_NOMOVE) return set_err(ctx, VMC_ERR_NOMOVE, "walker without an allowed move");
    if (st & VMC_DEV_INCONSISTENT) return set_err(ctx, VMC_ERR_ARG, "rate store inconsistent with walkers");
    if (st & VMC_DEV_TIMEOUT) return set_err(ctx, VMC_ERR_TIMEOUT, "a bounded device wait gave up");
    return VMC_OK;
}

vmc_status vmc_walkers_sizes(int W, int M, int na, int nb, const vmc_lists *L, int64_t out[10]) {
    if (!out || W < 0 || M < 1 || na < 0 || nb < 0 || na > M || nb > M) return VMC_ERR_ARG;
    const int64_t nw = (M + 31) / 32;
    out[0] = (int64_t)W * 2 * nw;
    out[1] = (int64_t)W * (na + nb);
    out[2] = (int64_t)W * (2 * M - na - nb);
    out[3] = (int64_t)W * 2 * M;
    out[4] = (int64_t)W * (int64_t)walker_stride_G(M, na, nb);
    out[5] = (int64_t)W * (int64_t)walker_stride_A(na, nb);
    out[6] = (int64_t)W * 2 * M;
    out[7] = (int64_t)W * 2 * (L ? (L->ns + 3) & ~(int64_t)3 : 0);
    out[8] = W;
    out[9] = W;
    return VMC_OK;
}

static vmc_status init_common(vmc_ctx *ctx, vmc_lists *L, const vmc_params *P, vmc_walkers *Wk, int full) {
    if (!ctx) return VMC_ERR_ARG;
    if (!L || !P || !P->J || !P->C_alpha || !P->C_beta) return set_err(ctx, VMC_ERR_ARG, "null lists or parameters");
    vmc_status st = check_walkers(ctx, Wk, L);
    if (st) return st;
    st = check_cps(ctx, P, Wk);
    if (st) return st;
    ctx->rates_valid = 0;
    st = launch_init_walkers(ctx, L, P, Wk, full);
    if (st) return st;
    return launch_cps_state(ctx, P, Wk);
}

vmc_status vmc_walkers_init(vmc_ctx *ctx, vmc_lists *L, const vmc_params *P, vmc_walkers *Wk) {
    return init_common(ctx, L, P, Wk, 1);
}

vmc_status vmc_walkers_refresh(vmc_ctx *ctx, vmc_lists *L, const vmc_params *P, vmc_walkers *Wk) {
    return init_common(ctx, L, P, Wk, 0);
}

vmc_status vmc_local_energy(vmc_ctx *ctx, const vmc_lists *Lc, const vmc_params *P, vmc_walkers *Wk,
                            double eps_run, double *e_loc, double *t_res) {
    if (!ctx) return VMC_ERR_ARG;
    vmc_lists *L = const_cast<vmc_lists *>(Lc);
    if (!L || !P || !e_loc || !t_res) return set_err(ctx, VMC_ERR_ARG, "null argument");
    vmc_status st = check_walkers(ctx, Wk, L);
    if (st) return st;
    if (!(eps_run >= L->eps_build)) return set_err(ctx, VMC_ERR_ARG, "eps_run must be >= the build eps");
    st = check_cps(ctx, P, Wk);
    if (st) return st;
    st = lists_set_eps(ctx, L, eps_run);
    if (st) return st;
    const int ng = L->view.n_groups;
    void *rates = nullptr;
    st = ensure_rates(ctx, sizeof(u128) * rate_store_units(Wk->W, ng), &rates);
    if (st) return st;
    st = launch_local_energy(ctx, L, Wk, cps_view(P), e_loc, t_res, (u128 *)rates, ng);
    if (st) return st;
    ctx->rates_walkers = Wk->G;
    ctx->rates_groups = ng;
    ctx->rates_valid = 1;
    return VMC_OK;
}

vmc_status vmc_ctmc_step(vmc_ctx *ctx, const vmc_lists *L, const vmc_params *P, vmc_walkers *Wk, uint64_t seed,
                         uint64_t *move_code) {
    if (!ctx) return VMC_ERR_ARG;
    if (!L || !P || !P->J || !move_code) return set_err(ctx, VMC_ERR_ARG, "null argument");
    vmc_status st = check_walkers(ctx, Wk, L);
    if (st) return st;
    if (!ctx->rates_valid || ctx->rates_walkers != Wk->G)
        return set_err(ctx, VMC_ERR_ARG, "vmc_local_energy must precede vmc_ctmc_step on the same walkers");
    st = check_cps(ctx, P, Wk);
    if (st) return st;
    st = launch_ctmc_step(ctx, L, P, Wk, seed, (const u128 *)ctx->rates, ctx->rates_groups, move_code);
    ctx->rates_valid = 0;
    return st;
}

vmc_status vmc_screened_moves(vmc_ctx *ctx, const vmc_lists *Lc, const vmc_params *P, const vmc_walkers *Wk,
                              double eps_run, int w_begin, int n_w, int64_t cap, uint64_t *code, double *ratio,
                              double *contrib, int64_t *count, int64_t *walked) {
    if (!ctx) return VMC_ERR_ARG;
    vmc_lists *L = const_cast<vmc_lists *>(Lc);
    if (!L || !P || !count) return set_err(ctx, VMC_ERR_ARG, "null argument");
    vmc_status st = check_walkers(ctx, Wk, L);
    if (st) return st;
    if (!(eps_run >= L->eps_build)) return set_err(ctx, VMC_ERR_ARG, "eps_run must be >= the build eps");
    if (w_begin < 0 || n_w < 1 || w_begin > Wk->W - n_w) return set_err(ctx, VMC_ERR_ARG, "walker range outside [0, W)");
    if (cap < 0 || (cap > 0 && (!code || !ratio || !contrib))) return set_err(ctx, VMC_ERR_ARG, "bad move buffers");
    st = check_cps(ctx, P, Wk);
    if (st) return st;
    if (L->eps_run != eps_run) ctx->rates_valid = 0;   // the stored rates belong to other list lengths
    st = lists_set_eps(ctx, L, eps_run);
    if (st) return st;
    return launch_screened_moves(ctx, L, Wk, cps_view(P), w_begin, n_w, cap, code, ratio, contrib, count, walked);
}

vmc_status vmc_local_energy_batch(vmc_ctx *ctx, int n, const vmc_batch_item *items) {
    if (!ctx) return VMC_ERR_ARG;
    for (int k = 0; items && k < n; ++k) {
        vmc_status st = check_walkers(ctx, items[k].walkers, items[k].lists);
        if (st) return st;
        if (items[k].params && items[k].params->cps)
            return set_err(ctx, VMC_ERR_ARG, "the batched launches do not take a correlator product");
    }
    ctx->rates_valid = 0;
    return launch_local_energy_batch(ctx, n, items);
}

vmc_status vmc_ctmc_step_batch(vmc_ctx *ctx, int n, const vmc_batch_item *items, uint64_t seed) {
    if (!ctx) return VMC_ERR_ARG;
    for (int k = 0; items && k < n; ++k) {
        vmc_status st = check_walkers(ctx, items[k].walkers, items[k].lists);
        if (st) return st;
        if (items[k].params && items[k].params->cps)
            return set_err(ctx, VMC_ERR_ARG, "the batched launches do not take a correlator product");
    }
    return launch_ctmc_step_batch(ctx, n, items, seed);
}

vmc_status vmc_autotune_local_energy(vmc_ctx *ctx, int n, const vmc_batch_item *items, int *threads_out) {
    if (!ctx) return VMC_ERR_ARG;
    const int cand[4] = {128, 256, 384, 512};
    float best = 1e30f;
    int pick = ctx->eloc_threads;
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess)
        return set_err(ctx, VMC_ERR_CUDA, "autotune events");
    // one item: time the per-system launch that item's caller makes; several: the batched launch
    auto run = [&]() -> vmc_status {
        if (n == 1 && items)
            return vmc_local_energy(ctx, items[0].lists, items[0].params, items[0].walkers, items[0].eps_run,
                                    items[0].d_e_loc, items[0].d_t_res);
        return vmc_local_energy_batch(ctx, n, items);
    };
    for (int c = 0; c < 4; ++c) {
        ctx->eloc_threads = cand[c];
        vmc_status st = run();                                         // warm-up
        if (st) { cudaEventDestroy(a); cudaEventDestroy(b); return st; }
        cudaEventRecord(a, ctx->stream);
        st = run();
        cudaEventRecord(b, ctx->stream);
        if (st) { cudaEventDestroy(a); cudaEventDestroy(b); return st; }
        cudaError_t e = cudaEventSynchronize(b);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (e != cudaSuccess) { cudaEventDestroy(a); cudaEventDestroy(b); return cuda_check(ctx, e, "autotune"); }
        if (ms < best) { best = ms; pick = cand[c]; }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    ctx->eloc_threads = pick;
    ctx->rates_batch.clear();
    if (threads_out) *threads_out = pick;
    return VMC_OK;
}

vmc_status vmc_grad_logpsi(vmc_ctx *ctx, const vmc_walkers *Wk, const double *w, double *dJ, double *dCa,
                           double *dCb) {
    if (!ctx) return VMC_ERR_ARG;
    vmc_status st = check_walkers(ctx, Wk, nullptr);
    if (st) return st;
    if (!w) return set_err(ctx, VMC_ERR_ARG, "null weights");
    if (!dJ && !(dCa && dCb)) return set_err(ctx, VMC_ERR_ARG, "no output");
    return launch_grad(ctx, Wk, w, dJ, dCa, dCb);
}

vmc_status vmc_accumulate_gradient(vmc_ctx *ctx, const vmc_walkers *Wk, const double *t, const double *e,
                                   double *aoJ, double *aoA, double *aoB, double *aeJ, double *aeA, double *aeB,
                                   double *sums) {
    if (!ctx) return VMC_ERR_ARG;
    vmc_status st = check_walkers(ctx, Wk, nullptr);
    if (st) return st;
    if (!t || !e || !aoJ || !aoA || !aoB || !aeJ || !aeA || !aeB || !sums)
        return set_err(ctx, VMC_ERR_ARG, "null argument");
    double *const o0[3] = {aoJ, aoA, aoB};
    double *const o1[3] = {aeJ, aeA, aeB};
    return launch_accumulate(ctx, Wk, t, e, o0, o1, sums);
}

vmc_status vmc_amsgrad_update(vmc_ctx *ctx, double *p, const double *g, double *m, double *n, size_t np,
                              double alpha, double b1, double b2) {
    if (!ctx) return VMC_ERR_ARG;
    if (np && (!p || !g || !m || !n)) return set_err(ctx, VMC_ERR_ARG, "null argument");
    return launch_amsgrad(ctx, p, g, m, n, np, alpha, b1, b2);
}

vmc_status vmc_energy_gradient(vmc_ctx *ctx, size_t n, const double *sums, const double *aO, const double *aEO,
                               double *g) {
    if (!ctx) return VMC_ERR_ARG;
    if (n && (!sums || !aO || !aEO || !g)) return set_err(ctx, VMC_ERR_ARG, "null argument");
    if (g == aO || g == aEO) return set_err(ctx, VMC_ERR_ARG, "g must not alias the sums");
    return launch_energy_gradient(ctx, n, sums, aO, aEO, g);
}

vmc_status vmc_walker_reduce(vmc_ctx *ctx, int W, const double *t, const double *e, double *out) {
    if (!ctx) return VMC_ERR_ARG;
    if (W < 1 || !t || !e || !out) return set_err(ctx, VMC_ERR_ARG, "bad argument");
    return launch_walker_reduce(ctx, W, t, e, out);
}

vmc_status vmc_log_psi(vmc_ctx *ctx, const vmc_walkers *Wk, const vmc_params *P, double *out) {
    if (!ctx) return VMC_ERR_ARG;
    vmc_status st = check_walkers(ctx, Wk, nullptr);
    if (st) return st;
    if (!P || !P->J || !P->C_alpha || !P->C_beta || !out) return set_err(ctx, VMC_ERR_ARG, "null argument");
    st = check_cps(ctx, P, Wk);
    if (st) return st;
    st = launch_log_psi(ctx, Wk, P, out);
    if (st) return st;
    return launch_cps_log_psi(ctx, P, Wk, out);
}

}  // extern "C"
