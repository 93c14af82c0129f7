// Screened integral lists in heat-bath form (Sec. II.A) and their per-entry Jastrow constants.
//
// Built once per eps on the host (O(M^4 log M), "the same cost as reading the integrals"),
// then copied to one device allocation.  Each walker's local energy walks, for every occupied
// pair, the pair's list sorted by |v| descending up to the first entry at or below eps_run; the
// cut position of every list for the current eps_run is precomputed (a binary search per list)
// so the kernels never test magnitudes.
//
// The host pass (build_host) needs no device: vmc_screened_lists_summary runs it alone and
// reports the list sizes, the near-tie count and a digest of every array the device copy is made
// from, so packed and dense integral input can be checked against each other without a GPU.
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

// Near tie of a screening magnitude x with the threshold: | |x| - eps | < 1e-12 max(1, eps).
// Such items could be kept or dropped by a rounding difference; they are counted, not resolved.
inline bool near_tie(double key, double eps) { return fabs(key - eps) < 1e-12 * (eps > 1.0 ? eps : 1.0); }

// (pq|rs) from dense [M^4] storage or from 8-fold packed storage: pair index pq = p(p+1)/2 + q
// for p >= q, element PQ(PQ+1)/2 + RS for PQ >= RS (M(M+1)/2 (M(M+1)/2 + 1)/2 doubles).
struct Eri {
    const double *d;
    size_t M;
    int packed;
    static size_t pair(size_t p, size_t q) { return p >= q ? p * (p + 1) / 2 + q : q * (q + 1) / 2 + p; }
    double operator()(int p, int q, int r, int s) const {
        if (!packed) return d[(((size_t)p * M + q) * M + r) * M + s];
        return d[pair(pair(p, q), pair(r, s))];
    }
};

// Everything the device copy of the lists is made from, built on the host.
struct HostLists {
    int M = 0;
    int64_t ns = 0, nds = 0, ndo = 0, ns_pad = 0;
    int64_t near_ties = 0;   // spin-orbital screening quantities within the near-tie band of eps
    int band = 0;
    std::vector<uint32_t> s_off, ds_off, do_off;
    std::vector<double> s_key, ds_key, do_key;
    std::vector<uint16_t> s_a;
    std::vector<uint32_t> s_owner, ds_ab, ds_owner, do_ab, do_owner;
    std::vector<double> ds_v, do_v;
    std::vector<double> Tj, Tjk, Jd, Kd, hd;
};

void pair_of_tri(int t, int M, int *p_out, int *q_out) {
    int p = 0;
    while (tri_index(p, M - 1, M) < t) ++p;
    *p_out = p;
    *q_out = t - tri_index(p, p + 1, M) + p + 1;
}

void build_host(int M, const double *h1, const Eri &E, double eps, HostLists &H) {
    const size_t MM = (size_t)M;
    const int npair = M * (M - 1) / 2;
    H.M = M;
    // ---- singles: S_ia = |h_ia| + sum_j |<ij|aj> - <ij|ja>| (same-spin j first, then the other);
    //      one spatial list serves both spins, so a near tie counts twice
    std::vector<std::vector<Ent>> sl(M);
    std::vector<int64_t> nt_s(M, 0);
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < M; ++i) {
        for (int a = 0; a < M; ++a) {
            if (a == i) continue;
            double acc = fabs(h1[(size_t)i * M + a]);
            for (int k = 0; k < M; ++k) acc += fabs(E(i, a, k, k) - E(i, k, k, a));
            for (int k = 0; k < M; ++k) acc += fabs(E(i, a, k, k) - 0.0);
            if (near_tie(acc, eps)) nt_s[i] += 2;
            if (acc > eps) sl[i].push_back(Ent{acc, acc, (uint16_t)a, 0});
        }
        std::sort(sl[i].begin(), sl[i].end(), ent_less);
    }
    // ---- same-spin doubles for p < q: v = (ap|bq) - (aq|bp), a < b, a,b not in {p,q} (both spins)
    std::vector<std::vector<Ent>> dl(npair > 0 ? npair : 0);
    std::vector<int64_t> nt_d(npair > 0 ? npair : 0, 0);
#pragma omp parallel for schedule(dynamic, 4)
    for (int t = 0; t < npair; ++t) {
        int p, q;
        pair_of_tri(t, M, &p, &q);
        std::vector<Ent> &v = dl[t];
        for (int a = 0; a < M; ++a) {
            if (a == p || a == q) continue;
            for (int b = a + 1; b < M; ++b) {
                if (b == p || b == q) continue;
                double x = E(a, p, b, q) - E(a, q, b, p);
                double key = fabs(x);
                if (near_tie(key, eps)) nt_d[t] += 2;
                if (key > eps) v.push_back(Ent{key, x, (uint16_t)a, (uint16_t)b});
            }
        }
        std::sort(v.begin(), v.end(), ent_less);
    }
    // ---- opposite-spin doubles (p alpha, q beta): v = (ap|bq), a != p, b != q
    std::vector<std::vector<Ent>> ol(MM * MM);
    std::vector<int64_t> nt_o(MM * MM, 0);
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
                if (near_tie(key, eps)) nt_o[t] += 1;
                if (key > eps) v.push_back(Ent{key, x, (uint16_t)a, (uint16_t)b});
            }
        }
        std::sort(v.begin(), v.end(), ent_less);
    }
    H.near_ties = 0;
    for (int64_t x : nt_s) H.near_ties += x;
    for (int64_t x : nt_d) H.near_ties += x;
    for (int64_t x : nt_o) H.near_ties += x;

    // ---- flatten
    H.s_off.assign(M + 1, 0);
    H.ds_off.assign(npair + 1, 0);
    H.do_off.assign(MM * MM + 1, 0);
    for (int i = 0; i < M; ++i) H.s_off[i + 1] = H.s_off[i] + (uint32_t)sl[i].size();
    for (int t = 0; t < npair; ++t) H.ds_off[t + 1] = H.ds_off[t] + (uint32_t)dl[t].size();
    for (size_t t = 0; t < MM * MM; ++t) H.do_off[t + 1] = H.do_off[t] + (uint32_t)ol[t].size();
    const int64_t ns = H.s_off[M], nds = H.ds_off[npair], ndo = H.do_off[MM * MM];
    H.ns = ns; H.nds = nds; H.ndo = ndo;
    H.s_key.assign(ns + 1, 0.0); H.ds_key.assign(nds + 1, 0.0); H.do_key.assign(ndo + 1, 0.0);
    H.s_a.assign(ns + 1, 0); H.s_owner.assign(ns + 1, 0);
    H.ds_ab.assign(nds + 1, 0); H.ds_owner.assign(nds + 1, 0); H.ds_v.assign(nds + 1, 0.0);
    H.do_ab.assign(ndo + 1, 0); H.do_owner.assign(ndo + 1, 0); H.do_v.assign(ndo + 1, 0.0);
    for (int i = 0; i < M; ++i)
        for (size_t k = 0; k < sl[i].size(); ++k) {
            const size_t e = H.s_off[i] + k;
            H.s_a[e] = sl[i][k].a;
            H.s_owner[e] = (uint32_t)i;
            H.s_key[e] = sl[i][k].key;
        }
    for (int t = 0; t < npair; ++t) {
        int p, q;
        pair_of_tri(t, M, &p, &q);
        for (size_t k = 0; k < dl[t].size(); ++k) {
            const size_t e = H.ds_off[t] + k;
            H.ds_ab[e] = (uint32_t)dl[t][k].a | ((uint32_t)dl[t][k].b << 16);
            H.ds_owner[e] = (uint32_t)p | ((uint32_t)q << 16);
            H.ds_v[e] = dl[t][k].v;
            H.ds_key[e] = dl[t][k].key;
        }
    }
    for (size_t t = 0; t < MM * MM; ++t)
        for (size_t k = 0; k < ol[t].size(); ++k) {
            const size_t e = H.do_off[t] + k;
            H.do_ab[e] = (uint32_t)ol[t][k].a | ((uint32_t)ol[t][k].b << 16);
            H.do_owner[e] = (uint32_t)(t / M) | ((uint32_t)(t % M) << 16);
            H.do_v[e] = ol[t][k].v;
            H.do_key[e] = ol[t][k].key;
        }
    // Fock-sum update tables and diagonal tables
    H.ns_pad = (ns + 3) & ~(int64_t)3;
    const int64_t ns_pad = H.ns_pad;
    H.Tj.assign(MM * (ns_pad + 1), 0.0); H.Tjk.assign(MM * (ns_pad + 1), 0.0);
    H.Jd.assign(MM * MM, 0.0); H.Kd.assign(MM * MM, 0.0); H.hd.assign(MM, 0.0);
    for (int64_t e = 0; e < ns; ++e) {
        const int i = (int)H.s_owner[e], a = H.s_a[e];
        for (int k = 0; k < M; ++k) {
            const double c = E(a, i, k, k);
            H.Tj[(size_t)k * ns_pad + e] = c;
            H.Tjk[(size_t)k * ns_pad + e] = c - E(a, k, k, i);
        }
    }
    for (int p = 0; p < M; ++p) {
        H.hd[p] = h1[(size_t)p * M + p];
        for (int q = 0; q < M; ++q) {
            H.Jd[(size_t)p * M + q] = E(p, p, q, q);
            H.Kd[(size_t)p * M + q] = E(p, q, q, p);
        }
    }
    // band of non-empty double lists: the largest |p - q| with a non-empty pair list
    int band = 0;
    for (int t = 0; t < npair; ++t)
        if (!dl[t].empty()) {
            int p, q;
            pair_of_tri(t, M, &p, &q);
            band = std::max(band, q - p);
        }
    for (size_t t = 0; t < MM * MM; ++t)
        if (!ol[t].empty()) band = std::max(band, std::abs((int)(t / M) - (int)(t % M)));
    H.band = band;
}

// FNV-1a over the bytes of a host array
template <typename T> void digest_add(uint64_t &h, const std::vector<T> &v) {
    const unsigned char *b = (const unsigned char *)v.data();
    for (size_t k = 0; k < v.size() * sizeof(T); ++k) {
        h ^= b[k];
        h *= 0x100000001B3ull;
    }
}

const char *check_build_args(int M, const double *h1, const double *eri, int eri_packed, double eps) {
    if (!h1 || !eri) return "null argument";
    if (M < 1 || M > VMC_MAX_M) return "M must be in [1, 256]";
    if (eri_packed != 0 && eri_packed != 1) return "eri_packed must be 0 or 1";
    if (!(eps >= 0.0)) return "eps must be >= 0";
    return nullptr;
}

}  // namespace

// The local energy's work units, [n_groups][32] in canonical move order.  Groups: singles blocks of
// 32 spin orbitals (unit = spin orbital i, list = singles(i)); then one group (or cpr chunks of 32
// candidates) per alpha spin-orbital row i, whose candidates j > i are the same-spin q in
// (p, p + band] followed by the opposite-spin q in [p - band, p + band]; then beta rows, rpg of them
// per group (lane = row offset x band + candidate) or cpr_b chunks each.  Groups and lanes run in
// ascending (i, j) order, which is the canonical order of the CTMC choice.
static void build_unit_table(const vmc_lists *L, const uint32_t *s_len, const uint32_t *ds_len,
                             const uint32_t *do_len, std::vector<uint4> &tab) {
    const ListsView &v = L->view;
    const int M = L->M, Gs = (2 * M + 31) / 32;
    tab.assign((size_t)v.n_groups * 32, make_uint4(0, 0, 0, 0));
    auto ncand = [&](int i) {   // candidates of spin-orbital row i
        const int sp = i >= M, p = i - sp * M, nS = std::min(v.band, M - 1 - p);
        return sp ? nS : nS + (std::min(M - 1, p + v.band) - std::max(0, p - v.band) + 1);
    };
    auto cand = [&](int i, int t) {
        const int sp = i >= M, p = i - sp * M, nS = std::min(v.band, M - 1 - p);
        return t < nS ? i + 1 + t : M + std::max(0, p - v.band) + (t - nS);
    };
    for (int g = 0; g < v.n_groups; ++g)
        for (int lane = 0; lane < 32; ++lane) {
            uint4 &e = tab[(size_t)g * 32 + lane];
            if (g < Gs) {
                const int i = g * 32 + lane;
                if (i >= 2 * M) continue;
                const int sp = i >= M, p = i - sp * M;
                e = make_uint4((uint32_t)p, L->h_s_off[p], s_len[p], (uint32_t)(sp << 2));
                continue;
            }
            const int ga = g - Gs;
            int i, t;
            if (ga < M * v.cpr) {
                i = ga / v.cpr;
                t = (ga % v.cpr) * 32 + lane;
            } else if (v.rpg > 1) {
                const int ro = lane / v.band;
                i = M + (ga - M * v.cpr) * v.rpg + ro;
                t = lane - ro * v.band;
                if (ro >= v.rpg || i >= 2 * M) continue;
            } else {
                const int gb = ga - M * v.cpr;
                i = M + gb / v.cpr_b;
                t = (gb % v.cpr_b) * 32 + lane;
            }
            if (t >= ncand(i)) continue;
            const int j = cand(i, t);
            const int si = i >= M, sj = j >= M, pi = i - si * M, pj = j - sj * M;
            if (si == sj) {
                const int tt = tri_index(pi, pj, M);
                e = make_uint4((uint32_t)pi | ((uint32_t)pj << 16), L->h_ds_off[tt], ds_len[tt], (uint32_t)(1 | (si << 2)));
            } else {
                const int tt = pi * M + pj;
                e = make_uint4((uint32_t)pi | ((uint32_t)pj << 16), L->h_do_off[tt], do_len[tt], 2u);
            }
        }
}

// Effective list lengths for eps_run (host binary searches, one small upload) and the unit table.
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
    std::vector<uint4> tab;
    build_unit_table(L, s_len.data(), ds_len.data(), do_len.data(), tab);
    cudaError_t e;
    e = cudaMemcpyAsync((void *)L->view.unit_tab, tab.data(), sizeof(uint4) * tab.size(), cudaMemcpyHostToDevice,
                        ctx->stream);
    if (e == cudaSuccess)
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

extern "C" vmc_status vmc_screened_lists_summary(int M, const double *h1, const double *eri, int eri_packed,
                                                 double eps, int64_t out[5]) {
    if (!out || check_build_args(M, h1, eri, eri_packed, eps)) return VMC_ERR_ARG;
    HostLists H;
    build_host(M, h1, Eri{eri, (size_t)M, eri_packed}, eps, H);
    uint64_t h = 0xCBF29CE484222325ull;
    digest_add(h, H.s_off); digest_add(h, H.ds_off); digest_add(h, H.do_off);
    digest_add(h, H.s_key); digest_add(h, H.ds_key); digest_add(h, H.do_key);
    digest_add(h, H.s_a); digest_add(h, H.s_owner);
    digest_add(h, H.ds_ab); digest_add(h, H.ds_owner); digest_add(h, H.ds_v);
    digest_add(h, H.do_ab); digest_add(h, H.do_owner); digest_add(h, H.do_v);
    digest_add(h, H.Tj); digest_add(h, H.Tjk); digest_add(h, H.Jd); digest_add(h, H.Kd); digest_add(h, H.hd);
    out[0] = H.ns; out[1] = H.nds; out[2] = H.ndo; out[3] = H.near_ties;
    out[4] = (int64_t)h;
    return VMC_OK;
}

extern "C" vmc_status vmc_build_screened_lists(vmc_ctx *ctx, int M, const double *h1, const double *eri,
                                               int eri_packed, double e_core, double eps, vmc_lists **out) {
    if (!ctx || !out) return ctx ? set_err(ctx, VMC_ERR_ARG, "null argument") : VMC_ERR_ARG;
    if (const char *why = check_build_args(M, h1, eri, eri_packed, eps)) return set_err(ctx, VMC_ERR_ARG, why);
    *out = nullptr;
    const size_t MM = (size_t)M;
    const int npair = M * (M - 1) / 2;
    HostLists H;
    build_host(M, h1, Eri{eri, MM, eri_packed}, eps, H);
    const int64_t ns = H.ns, nds = H.nds, ndo = H.ndo, ns_pad = H.ns_pad;
    if (ns >= (int64_t)1 << 27 || nds >= (int64_t)1 << 27 || ndo >= (int64_t)1 << 27)
        return set_err(ctx, VMC_ERR_ARG, "more than 2^27 entries in one list class");

    vmc_lists *L = new vmc_lists();
    L->M = M;
    L->eps_build = eps;
    L->near_ties_build = H.near_ties;
    L->ns = ns; L->nds = nds; L->ndo = ndo;
    auto dup_u32 = [](const std::vector<uint32_t> &v) {
        uint32_t *p = (uint32_t *)malloc(sizeof(uint32_t) * v.size());
        memcpy(p, v.data(), sizeof(uint32_t) * v.size());
        return p;
    };
    auto dup_f64 = [](const std::vector<double> &v) {
        double *p = (double *)malloc(sizeof(double) * v.size());
        memcpy(p, v.data(), sizeof(double) * v.size());
        return p;
    };
    L->h_s_off = dup_u32(H.s_off); L->h_ds_off = dup_u32(H.ds_off); L->h_do_off = dup_u32(H.do_off);
    L->h_s_key = dup_f64(H.s_key); L->h_ds_key = dup_f64(H.ds_key); L->h_do_key = dup_f64(H.do_key);

    // packed per-entry records (the Jastrow constants are rewritten by every refresh)
    std::vector<float4> s_r32(ns + 1), ds_r32(nds + 1), do_r32(ndo + 1);
    std::vector<double4_32a> s_r64(ns + 1), ds_r64(nds + 1), do_r64(ndo + 1);
    auto bits_d = [](uint32_t u) { double d = 0.0; uint64_t x = u; memcpy(&d, &x, 8); return d; };
    auto bits_f = [](uint32_t u) { float f; memcpy(&f, &u, 4); return f; };
    for (int64_t e = 0; e < ns; ++e) {
        s_r32[e] = make_float4(bits_f(H.s_a[e]), 1.0f, 1.0f, 0.0f);
        s_r64[e] = make_double4_32a(bits_d(H.s_a[e]), 1.0, 1.0, 0.0);
    }
    for (int64_t e = 0; e < nds; ++e) {
        ds_r32[e] = make_float4(bits_f(H.ds_ab[e]), (float)H.ds_v[e], 1.0f, 1.0f);
        ds_r64[e] = make_double4_32a(bits_d(H.ds_ab[e]), H.ds_v[e], 1.0, 1.0);
    }
    for (int64_t e = 0; e < ndo; ++e) {
        do_r32[e] = make_float4(bits_f(H.do_ab[e]), (float)H.do_v[e], 1.0f, 0.0f);
        do_r64[e] = make_double4_32a(bits_d(H.do_ab[e]), H.do_v[e], 1.0, 0.0);
    }
    std::vector<float> Tjf(MM * (ns_pad + 1)), Tjkf(MM * (ns_pad + 1));
    for (size_t k = 0; k < Tjf.size(); ++k) {
        Tjf[k] = (float)H.Tj[k];
        Tjkf[k] = (float)H.Tjk[k];
    }

    // ---- work-unit geometry (see build_unit_table)
    ListsView &v = L->view;
    v.M = M; v.ns = ns; v.nds = nds; v.ndo = ndo; v.e_core = e_core; v.ns_pad = ns_pad;
    {
        const int band = H.band;
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

    // ---- one device allocation
    struct Piece { const void *src; size_t bytes; size_t off; };
    std::vector<Piece> pcs;
    size_t off = 0;
    auto add = [&](const void *src, size_t bytes) {
        pcs.push_back(Piece{src, bytes, off});
        off = align256(off + (bytes ? bytes : 1));
        return pcs.size() - 1;
    };
    const size_t i_s_off = add(H.s_off.data(), sizeof(uint32_t) * (M + 1));
    const size_t i_s_len = add(nullptr, sizeof(uint32_t) * M);
    const size_t i_s_owner = add(H.s_owner.data(), sizeof(uint32_t) * ns);
    const size_t i_s_a = add(H.s_a.data(), sizeof(uint16_t) * ns);
    const size_t i_s_r32 = add(s_r32.data(), sizeof(float4) * ns);
    const size_t i_s_r64 = add(s_r64.data(), sizeof(double4_32a) * ns);
    const size_t i_ds_off = add(H.ds_off.data(), sizeof(uint32_t) * (npair + 1));
    const size_t i_ds_len = add(nullptr, sizeof(uint32_t) * (npair > 0 ? npair : 1));
    const size_t i_ds_ab = add(H.ds_ab.data(), sizeof(uint32_t) * nds);
    const size_t i_ds_owner = add(H.ds_owner.data(), sizeof(uint32_t) * nds);
    const size_t i_ds_r32 = add(ds_r32.data(), sizeof(float4) * nds);
    const size_t i_ds_r64 = add(ds_r64.data(), sizeof(double4_32a) * nds);
    const size_t i_do_off = add(H.do_off.data(), sizeof(uint32_t) * (MM * MM + 1));
    const size_t i_do_len = add(nullptr, sizeof(uint32_t) * MM * MM);
    const size_t i_do_ab = add(H.do_ab.data(), sizeof(uint32_t) * ndo);
    const size_t i_do_owner = add(H.do_owner.data(), sizeof(uint32_t) * ndo);
    const size_t i_do_r32 = add(do_r32.data(), sizeof(float4) * ndo);
    const size_t i_do_r64 = add(do_r64.data(), sizeof(double4_32a) * ndo);
    const size_t i_Tj = add(H.Tj.data(), sizeof(double) * MM * ns_pad);
    const size_t i_Tjk = add(H.Tjk.data(), sizeof(double) * MM * ns_pad);
    const size_t i_Tjf = add(Tjf.data(), sizeof(float) * MM * ns_pad);
    const size_t i_Tjkf = add(Tjkf.data(), sizeof(float) * MM * ns_pad);
    const size_t i_Jd = add(H.Jd.data(), sizeof(double) * MM * MM);
    const size_t i_Kd = add(H.Kd.data(), sizeof(double) * MM * MM);
    const size_t i_hd = add(H.hd.data(), sizeof(double) * MM);
    const size_t i_h1 = add(h1, sizeof(double) * MM * MM);
    const size_t i_cf = add(nullptr, sizeof(float) * MM * 2 * MM);
    const size_t i_cdig = add(nullptr, g_ozaki_table_bytes((int)MM));
    const size_t i_jsym = add(nullptr, (sizeof(double) + sizeof(float)) * 4 * MM * MM);
    const size_t i_tab = add(nullptr, sizeof(uint4) * 32 * (size_t)v.n_groups);

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
    v.unit_tab = (const uint4 *)P(i_tab);
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
    L->cdig = P(i_cdig);
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

extern "C" vmc_status vmc_lists_layout(const vmc_lists *L, int *band, int *n_groups) {
    if (!L) return VMC_ERR_ARG;
    if (band) *band = L->view.band;
    if (n_groups) *n_groups = L->view.n_groups;
    return VMC_OK;
}

extern "C" vmc_status vmc_lists_near_ties(const vmc_lists *L, double eps, int64_t *n_near) {
    if (!L || !n_near || !(eps >= 0.0)) return VMC_ERR_ARG;
    if (eps == L->eps_build) {   // counted by the builder over every candidate, kept or not
        *n_near = L->near_ties_build;
        return VMC_OK;
    }
    // above the build threshold every candidate within the band is a stored entry
    if (!(eps - 1e-12 * (eps > 1.0 ? eps : 1.0) > L->eps_build)) return VMC_ERR_ARG;
    const int M = L->M, npair = M * (M - 1) / 2;
    int64_t n = 0;
    for (int64_t e = 0; e < L->ns; ++e) n += near_tie(L->h_s_key[e], eps) ? 2 : 0;
    for (int64_t e = 0; e < L->nds; ++e) n += near_tie(L->h_ds_key[e], eps) ? 2 : 0;
    for (int64_t e = 0; e < L->ndo; ++e) n += near_tie(L->h_do_key[e], eps) ? 1 : 0;
    (void)npair;
    *n_near = n;
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
