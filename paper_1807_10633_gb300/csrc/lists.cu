// Screened integral lists in heat-bath form (Sec. II.A) and their per-entry Jastrow constants.
//
// Built once per eps on the host (O(M^4 log M), "the same cost as reading the integrals"),
// then copied to one device allocation.  Each walker's local energy walks, for every occupied
// pair, the pair's list sorted by |v| descending up to the first entry at or below eps_run; the
// cut position of every list for the current eps_run is precomputed (a binary search per list)
// so the kernels never test magnitudes.
#include <math.h>
#include <omp.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cstdlib>
#include <vector>

#include "common.cuh"

namespace {

struct Ent {
    double key;
    double v;
    uint16_t a, b;
};

bool ent_less(const Ent &x, const Ent &y) {   // |v| descending, then a, then b ascending
    if (x.key != y.key) return x.key > y.key;
    if (x.a != y.a) return x.a < y.a;
    return x.b < y.b;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

uint32_t count_above(const double *key, uint32_t n, double eps) {   // keys sorted descending
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        uint32_t mid = (lo + hi) / 2;
        if (key[mid] > eps) lo = mid + 1; else hi = mid;
    }
    return lo;
}

}  // namespace

// Effective list lengths for eps_run (host binary searches, one small upload).
vmc_status lists_set_eps(vmc_ctx *ctx, vmc_lists *L, double eps_run) {
    if (L->eps_run == eps_run) return VMC_OK;
    const int M = L->M;
    const int npair = M * (M - 1) / 2;
    std::vector<uint32_t> s_len(M), ds_len(npair > 0 ? npair : 1), do_len((size_t)M * M);
    for (int i = 0; i < M; ++i)
        s_len[i] = count_above(L->h_s_key + L->h_s_off[i], L->h_s_off[i + 1] - L->h_s_off[i], eps_run);
    for (int t = 0; t < npair; ++t)
        ds_len[t] = count_above(L->h_ds_key + L->h_ds_off[t], L->h_ds_off[t + 1] - L->h_ds_off[t], eps_run);
    for (int t = 0; t < M * M; ++t)
        do_len[t] = count_above(L->h_do_key + L->h_do_off[t], L->h_do_off[t + 1] - L->h_do_off[t], eps_run);
    cudaError_t e;
    e = cudaMemcpyAsync((void *)L->view.s_len, s_len.data(), sizeof(uint32_t) * M, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess && npair > 0)
        e = cudaMemcpyAsync((void *)L->view.ds_len, ds_len.data(), sizeof(uint32_t) * npair, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync((void *)L->view.do_len, do_len.data(), sizeof(uint32_t) * M * M, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);   // host vectors go out of scope
    if (e != cudaSuccess) return cuda_check(ctx, e, "uploading list lengths");
    L->eps_run = eps_run;
    return VMC_OK;
}

extern "C" vmc_status vmc_build_screened_lists(vmc_ctx *ctx, int M, const double *h1, const double *eri,
                                               double e_core, double eps, vmc_lists **out) {
    if (!ctx || !out || !h1 || !eri) return ctx ? set_err(ctx, VMC_ERR_ARG, "null argument") : VMC_ERR_ARG;
    if (M < 1 || M > VMC_MAX_M) return set_err(ctx, VMC_ERR_ARG, "M must be in [1, 256]");
    if (!(eps >= 0.0)) return set_err(ctx, VMC_ERR_ARG, "eps must be >= 0");
    *out = nullptr;
    const size_t MM = (size_t)M;
    auto E = [&](int p, int q, int r, int s) { return eri[((p * MM + q) * MM + r) * MM + s]; };
    const int npair = M * (M - 1) / 2;

    // ---- singles: S_ia = |h_ia| + sum_j |<ij|aj> - <ij|ja>| (same-spin j first, then the other)
    std::vector<std::vector<Ent>> sl(M);
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < M; ++i) {
        for (int a = 0; a < M; ++a) {
            if (a == i) continue;
            double acc = fabs(h1[(size_t)i * M + a]);
            for (int k = 0; k < M; ++k) acc += fabs(E(i, a, k, k) - E(i, k, k, a));
            for (int k = 0; k < M; ++k) acc += fabs(E(i, a, k, k) - 0.0);
            if (acc > eps) sl[i].push_back(Ent{acc, acc, (uint16_t)a, 0});
        }
        std::sort(sl[i].begin(), sl[i].end(), ent_less);
    }
    // ---- same-spin doubles for p < q: v = (ap|bq) - (aq|bp), a < b, a,b not in {p,q}
    std::vector<std::vector<Ent>> dl(npair > 0 ? npair : 0);
#pragma omp parallel for schedule(dynamic, 4)
    for (int t = 0; t < npair; ++t) {
        int p = 0;
        while (tri_index(p, M - 1, M) < t) ++p;
        int q = t - tri_index(p, p + 1, M) + p + 1;
        std::vector<Ent> &v = dl[t];
        for (int a = 0; a < M; ++a) {
            if (a == p || a == q) continue;
            for (int b = a + 1; b < M; ++b) {
                if (b == p || b == q) continue;
                double x = E(a, p, b, q) - E(a, q, b, p);
                double key = fabs(x);
                if (key > eps) v.push_back(Ent{key, x, (uint16_t)a, (uint16_t)b});
            }
        }
        std::sort(v.begin(), v.end(), ent_less);
    }
    // ---- opposite-spin doubles (p alpha, q beta): v = (ap|bq), a != p, b != q
    std::vector<std::vector<Ent>> ol(MM * MM);
#pragma omp parallel for schedule(dynamic, 4)
    for (int t = 0; t < M * M; ++t) {
        const int p = t / M, q = t % M;
        std::vector<Ent> &v = ol[t];
        for (int a = 0; a < M; ++a) {
            if (a == p) continue;
            for (int b = 0; b < M; ++b) {
                if (b == q) continue;
                double x = E(a, p, b, q) - 0.0;
                double key = fabs(x);
                if (key > eps) v.push_back(Ent{key, x, (uint16_t)a, (uint16_t)b});
            }
        }
        std::sort(v.begin(), v.end(), ent_less);
    }

    // ---- flatten
    vmc_lists *L = new vmc_lists();
    L->M = M;
    L->eps_build = eps;
    L->h_s_off = (uint32_t *)calloc(M + 1, sizeof(uint32_t));
    L->h_ds_off = (uint32_t *)calloc(npair + 1, sizeof(uint32_t));
    L->h_do_off = (uint32_t *)calloc(MM * MM + 1, sizeof(uint32_t));
    for (int i = 0; i < M; ++i) L->h_s_off[i + 1] = L->h_s_off[i] + (uint32_t)sl[i].size();
    for (int t = 0; t < npair; ++t) L->h_ds_off[t + 1] = L->h_ds_off[t] + (uint32_t)dl[t].size();
    for (size_t t = 0; t < MM * MM; ++t) L->h_do_off[t + 1] = L->h_do_off[t] + (uint32_t)ol[t].size();
    const int64_t ns = L->h_s_off[M], nds = L->h_ds_off[npair], ndo = L->h_do_off[MM * MM];
    if (ns >= (int64_t)1 << 27 || nds >= (int64_t)1 << 27 || ndo >= (int64_t)1 << 27) {
        vmc_lists_destroy(L);
        return set_err(ctx, VMC_ERR_ARG, "more than 2^27 entries in one list class");
    }
    L->ns = ns; L->nds = nds; L->ndo = ndo;
    L->h_s_key = (double *)malloc(sizeof(double) * (ns + 1));
    L->h_ds_key = (double *)malloc(sizeof(double) * (nds + 1));
    L->h_do_key = (double *)malloc(sizeof(double) * (ndo + 1));

    std::vector<uint16_t> s_a(ns + 1);
    std::vector<uint32_t> s_owner(ns + 1), ds_ab(nds + 1), ds_owner(nds + 1), do_ab(ndo + 1), do_owner(ndo + 1);
    std::vector<double> ds_vd(nds + 1), do_vd(ndo + 1);
    for (int i = 0; i < M; ++i)
        for (size_t k = 0; k < sl[i].size(); ++k) {
            const size_t e = L->h_s_off[i] + k;
            s_a[e] = sl[i][k].a;
            s_owner[e] = (uint32_t)i;
            L->h_s_key[e] = sl[i][k].key;
        }
    for (int t = 0; t < npair; ++t) {
        int p = 0;
        while (tri_index(p, M - 1, M) < t) ++p;
        int q = t - tri_index(p, p + 1, M) + p + 1;
        for (size_t k = 0; k < dl[t].size(); ++k) {
            const size_t e = L->h_ds_off[t] + k;
            ds_ab[e] = (uint32_t)dl[t][k].a | ((uint32_t)dl[t][k].b << 16);
            ds_owner[e] = (uint32_t)p | ((uint32_t)q << 16);
            ds_vd[e] = dl[t][k].v;
            L->h_ds_key[e] = dl[t][k].key;
        }
    }
    for (size_t t = 0; t < MM * MM; ++t)
        for (size_t k = 0; k < ol[t].size(); ++k) {
            const size_t e = L->h_do_off[t] + k;
            do_ab[e] = (uint32_t)ol[t][k].a | ((uint32_t)ol[t][k].b << 16);
            do_owner[e] = (uint32_t)(t / M) | ((uint32_t)(t % M) << 16);
            do_vd[e] = ol[t][k].v;
            L->h_do_key[e] = ol[t][k].key;
        }
    // packed per-entry records (the Jastrow constants are rewritten by every refresh)
    std::vector<float4> s_r32(ns + 1), ds_r32(nds + 1), do_r32(ndo + 1);
    std::vector<double4_32a> s_r64(ns + 1), ds_r64(nds + 1), do_r64(ndo + 1);
    auto bits_d = [](uint32_t u) { double d = 0.0; uint64_t x = u; memcpy(&d, &x, 8); return d; };
    auto bits_f = [](uint32_t u) { float f; memcpy(&f, &u, 4); return f; };
    for (int64_t e = 0; e < ns; ++e) {
        s_r32[e] = make_float4(bits_f(s_a[e]), 1.0f, 1.0f, 0.0f);
        s_r64[e] = make_double4_32a(bits_d(s_a[e]), 1.0, 1.0, 0.0);
    }
    for (int64_t e = 0; e < nds; ++e) {
        ds_r32[e] = make_float4(bits_f(ds_ab[e]), (float)ds_vd[e], 1.0f, 1.0f);
        ds_r64[e] = make_double4_32a(bits_d(ds_ab[e]), ds_vd[e], 1.0, 1.0);
    }
    for (int64_t e = 0; e < ndo; ++e) {
        do_r32[e] = make_float4(bits_f(do_ab[e]), (float)do_vd[e], 1.0f, 0.0f);
        do_r64[e] = make_double4_32a(bits_d(do_ab[e]), do_vd[e], 1.0, 0.0);
    }
    // Fock tables and diagonal tables
    const int64_t ns_pad = (ns + 3) & ~(int64_t)3;
    std::vector<double> Tj(MM * (ns_pad + 1)), Tjk(MM * (ns_pad + 1)), Jd(MM * MM), Kd(MM * MM), hd(MM);
    std::vector<float> Tjf(MM * (ns_pad + 1)), Tjkf(MM * (ns_pad + 1));
    for (int64_t e = 0; e < ns; ++e) {
        const int i = (int)s_owner[e], a = s_a[e];
        for (int k = 0; k < M; ++k) {
            const double c = E(a, i, k, k);
            Tj[(size_t)k * ns_pad + e] = c;
            Tjk[(size_t)k * ns_pad + e] = c - E(a, k, k, i);
            Tjf[(size_t)k * ns_pad + e] = (float)Tj[(size_t)k * ns_pad + e];
            Tjkf[(size_t)k * ns_pad + e] = (float)Tjk[(size_t)k * ns_pad + e];
        }
    }
    for (int p = 0; p < M; ++p) {
        hd[p] = h1[(size_t)p * M + p];
        for (int q = 0; q < M; ++q) {
            Jd[(size_t)p * M + q] = E(p, p, q, q);
            Kd[(size_t)p * M + q] = E(p, q, q, p);
        }
    }

    // ---- one device allocation
    struct Piece { const void *src; size_t bytes; size_t off; };
    std::vector<Piece> pcs;
    size_t off = 0;
    auto add = [&](const void *src, size_t bytes) {
        pcs.push_back(Piece{src, bytes, off});
        off = align256(off + (bytes ? bytes : 1));
        return pcs.size() - 1;
    };
    const size_t i_s_off = add(L->h_s_off, sizeof(uint32_t) * (M + 1));
    const size_t i_s_len = add(nullptr, sizeof(uint32_t) * M);
    const size_t i_s_owner = add(s_owner.data(), sizeof(uint32_t) * ns);
    const size_t i_s_a = add(s_a.data(), sizeof(uint16_t) * ns);
    const size_t i_s_r32 = add(s_r32.data(), sizeof(float4) * ns);
    const size_t i_s_r64 = add(s_r64.data(), sizeof(double4_32a) * ns);
    const size_t i_ds_off = add(L->h_ds_off, sizeof(uint32_t) * (npair + 1));
    const size_t i_ds_len = add(nullptr, sizeof(uint32_t) * (npair > 0 ? npair : 1));
    const size_t i_ds_ab = add(ds_ab.data(), sizeof(uint32_t) * nds);
    const size_t i_ds_owner = add(ds_owner.data(), sizeof(uint32_t) * nds);
    const size_t i_ds_r32 = add(ds_r32.data(), sizeof(float4) * nds);
    const size_t i_ds_r64 = add(ds_r64.data(), sizeof(double4_32a) * nds);
    const size_t i_do_off = add(L->h_do_off, sizeof(uint32_t) * (MM * MM + 1));
    const size_t i_do_len = add(nullptr, sizeof(uint32_t) * MM * MM);
    const size_t i_do_ab = add(do_ab.data(), sizeof(uint32_t) * ndo);
    const size_t i_do_owner = add(do_owner.data(), sizeof(uint32_t) * ndo);
    const size_t i_do_r32 = add(do_r32.data(), sizeof(float4) * ndo);
    const size_t i_do_r64 = add(do_r64.data(), sizeof(double4_32a) * ndo);
    const size_t i_Tj = add(Tj.data(), sizeof(double) * MM * ns_pad);
    const size_t i_Tjk = add(Tjk.data(), sizeof(double) * MM * ns_pad);
    const size_t i_Tjf = add(Tjf.data(), sizeof(float) * MM * ns_pad);
    const size_t i_Tjkf = add(Tjkf.data(), sizeof(float) * MM * ns_pad);
    const size_t i_Jd = add(Jd.data(), sizeof(double) * MM * MM);
    const size_t i_Kd = add(Kd.data(), sizeof(double) * MM * MM);
    const size_t i_hd = add(hd.data(), sizeof(double) * MM);
    const size_t i_h1 = add(h1, sizeof(double) * MM * MM);
    const size_t i_cf = add(nullptr, sizeof(float) * MM * 2 * MM);
    const size_t i_jsym = add(nullptr, (sizeof(double) + sizeof(float)) * 4 * MM * MM);

    cudaError_t ce = cudaSetDevice(ctx->device);
    if (ce == cudaSuccess) ce = cudaMalloc(&L->dev, off);
    if (ce != cudaSuccess) {
        vmc_lists_destroy(L);
        return set_err(ctx, VMC_ERR_OOM, std::string("cudaMalloc lists: ") + cudaGetErrorString(ce));
    }
    L->dev_bytes = off;
    char *base = (char *)L->dev;
    for (const Piece &p : pcs) {
        if (!p.src || !p.bytes) continue;
        ce = cudaMemcpy(base + p.off, p.src, p.bytes, cudaMemcpyHostToDevice);
        if (ce != cudaSuccess) {
            vmc_lists_destroy(L);
            return cuda_check(ctx, ce, "uploading lists");
        }
    }
    auto P = [&](size_t idx) { return (void *)(base + pcs[idx].off); };
    ListsView &v = L->view;
    v.M = M; v.ns = ns; v.nds = nds; v.ndo = ndo; v.e_core = e_core; v.ns_pad = ns_pad;
    {
        int band = 0;
        for (int t = 0; t < npair; ++t)
            if (!dl[t].empty()) {
                int p = 0;
                while (tri_index(p, M - 1, M) < t) ++p;
                const int q = t - tri_index(p, p + 1, M) + p + 1;
                band = std::max(band, q - p);
            }
        for (size_t t = 0; t < MM * MM; ++t)
            if (!ol[t].empty()) band = std::max(band, std::abs((int)(t / M) - (int)(t % M)));
        // candidates of an alpha row: same-spin q in (p, p+band], opposite q in [p-band, p+band];
        // no row groups at all when every double list is empty (e.g. the Hubbard model)
        bool any_double = nds > 0 || ndo > 0;
        const int cand = std::min(band, M - 1) + std::min(2 * band + 1, M);
        v.band = band;
        v.cpr = any_double ? std::max(1, (cand + 31) / 32) : 0;
        // beta rows have at most `band` candidates: 32 / band of them share one warp group
        v.rpg = (band >= 1 && band <= 32) ? 32 / band : 1;
        v.cpr_b = band <= 32 ? 1 : (band + 31) / 32;
        const int nb_groups = (!any_double || band == 0) ? 0 : (v.rpg > 1 ? (M + v.rpg - 1) / v.rpg : M * v.cpr_b);
        v.n_groups = (2 * M + 31) / 32 + M * v.cpr + nb_groups;
    }
    v.s_off = (const uint32_t *)P(i_s_off); v.s_len = (const uint32_t *)P(i_s_len);
    v.s_owner = (const uint32_t *)P(i_s_owner); v.s_a = (const uint16_t *)P(i_s_a);
    v.s_rec32 = (const float4 *)P(i_s_r32); v.s_rec64 = (const double4_32a *)P(i_s_r64);
    v.ds_off = (const uint32_t *)P(i_ds_off); v.ds_len = (const uint32_t *)P(i_ds_len);
    v.ds_ab = (const uint32_t *)P(i_ds_ab); v.ds_owner = (const uint32_t *)P(i_ds_owner);
    v.ds_rec32 = (const float4 *)P(i_ds_r32); v.ds_rec64 = (const double4_32a *)P(i_ds_r64);
    v.do_off = (const uint32_t *)P(i_do_off); v.do_len = (const uint32_t *)P(i_do_len);
    v.do_ab = (const uint32_t *)P(i_do_ab); v.do_owner = (const uint32_t *)P(i_do_owner);
    v.do_rec32 = (const float4 *)P(i_do_r32); v.do_rec64 = (const double4_32a *)P(i_do_r64);
    v.Tj = (const double *)P(i_Tj); v.Tjk = (const double *)P(i_Tjk);
    v.Tjf = (const float *)P(i_Tjf); v.Tjkf = (const float *)P(i_Tjkf);
    v.Jd = (const double *)P(i_Jd); v.Kd = (const double *)P(i_Kd);
    v.hd = (const double *)P(i_hd); v.h1 = (const double *)P(i_h1);
    L->cf = P(i_cf);
    L->jsym = P(i_jsym);
    // the Jastrow constants are written by the first walker (re)initialisation
    vmc_status st = lists_set_eps(ctx, L, eps);
    if (st != VMC_OK) { vmc_lists_destroy(L); return st; }
    *out = L;
    return VMC_OK;
}

extern "C" vmc_status vmc_lists_destroy(vmc_lists *L) {
    if (!L) return VMC_OK;
    if (L->dev) cudaFree(L->dev);
    free(L->h_s_key); free(L->h_ds_key); free(L->h_do_key);
    free(L->h_s_off); free(L->h_ds_off); free(L->h_do_off);
    delete L;
    return VMC_OK;
}

extern "C" vmc_status vmc_lists_info(const vmc_lists *L, int64_t *ns, int64_t *nds, int64_t *ndo) {
    if (!L) return VMC_ERR_ARG;
    if (ns) *ns = L->ns;
    if (nds) *nds = L->nds;
    if (ndo) *ndo = L->ndo;
    return VMC_OK;
}

// ------------------------------------------------------------------ Jastrow constants
// For a move n -> m the pair-Jastrow ratio is exp(S_a + S_b - S_i - S_j) times a factor that
// depends only on the four spin orbitals and J:
//   w = exp(-J_ai - J_aj - J_bi - J_bj + J_ab + J_ij + d_a + d_b - d_i - d_j)   (doubles)
//   w = exp(-J_ai + d_a - d_i)                                                   (singles)
// with S_p = sum_{k occ, k != p} J_pk and d_p = J_pp.  These w are stored with every list entry.
__global__ void k_refresh_jastrow(ListsView L, const double *__restrict__ J, double *__restrict__ js64,
                                  float *__restrict__ js32) {
    const int M = L.M, N2 = 2 * M;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < N2 * N2; t += gridDim.x * blockDim.x) {
        const double v = jget(J, N2, t / N2, t % N2);   // symmetric copies for row-wise reads
        js64[t] = v;
        js32[t] = (float)v;
    }
    const int64_t tot = 2 * L.ns + 2 * L.nds + L.ndo;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
         t += (int64_t)gridDim.x * blockDim.x) {
        double lw;
        if (t < 2 * L.ns) {
            const int sg = (int)(t / L.ns);
            const int64_t e = t % L.ns;
            const int I = sg * M + (int)L.s_owner[e], A = sg * M + L.s_a[e];
            lw = -jget(J, N2, A, I) + jget(J, N2, A, A) - jget(J, N2, I, I);
            const double w = exp(lw);
            ((double *)&L.s_rec64[e])[1 + sg] = w;
            ((float *)&L.s_rec32[e])[1 + sg] = (float)w;
            continue;
        }
        int I, Jj, A, B;
        int64_t e;
        int cls;
        if (t < 2 * L.ns + 2 * L.nds) {
            const int64_t u = t - 2 * L.ns;
            cls = (int)(u / L.nds);
            e = u % L.nds;
            const uint32_t ow = L.ds_owner[e], ab = L.ds_ab[e];
            I = cls * M + (int)(ow & 0xFFFF); Jj = cls * M + (int)(ow >> 16);
            A = cls * M + (int)(ab & 0xFFFF); B = cls * M + (int)(ab >> 16);
        } else {
            cls = 2;
            e = t - 2 * L.ns - 2 * L.nds;
            const uint32_t ow = L.do_owner[e], ab = L.do_ab[e];
            I = (int)(ow & 0xFFFF); Jj = M + (int)(ow >> 16);
            A = (int)(ab & 0xFFFF); B = M + (int)(ab >> 16);
        }
        lw = -jget(J, N2, A, I) - jget(J, N2, A, Jj) - jget(J, N2, B, I) - jget(J, N2, B, Jj)
             + jget(J, N2, A, B) + jget(J, N2, I, Jj)
             + jget(J, N2, A, A) + jget(J, N2, B, B) - jget(J, N2, I, I) - jget(J, N2, Jj, Jj);
        const double w = exp(lw);
        if (cls < 2) {
            ((double *)&L.ds_rec64[e])[2 + cls] = w;
            ((float *)&L.ds_rec32[e])[2 + cls] = (float)w;
        } else {
            ((double *)&L.do_rec64[e])[2] = w;
            ((float *)&L.do_rec32[e])[2] = (float)w;
        }
    }
}

vmc_status launch_refresh_jastrow(vmc_ctx *ctx, vmc_lists *L, const double *J) {
    const int64_t tot = std::max<int64_t>(2 * L->ns + 2 * L->nds + L->ndo, 4 * (int64_t)L->M * L->M);
    int blocks = (int)std::min<int64_t>((tot + 255) / 256, 152 * 16);
    double *js64 = (double *)L->jsym;
    float *js32 = (float *)(js64 + 4 * (size_t)L->M * L->M);
    k_refresh_jastrow<<<blocks, 256, 0, ctx->stream>>>(L->view, J, js64, js32);
    ctx->launches += 1;
    return cuda_check(ctx, cudaGetLastError(), "k_refresh_jastrow");
}
