// Screened local energy (Sec. II.A, Eq. eloc:hci) and the rejection-free CTMC move (Sec. II.B).
//
// One CTA per walker.  The walker's G (virtual rows only), exp(S) and the orbital -> column /
// slot map are staged in shared memory; the screened lists (shared by all walkers, L2-resident)
// are streamed per occupied pair.  Work is split into "groups" in canonical move order:
//   singles : blocks of 32 consecutive spin orbitals i; unit = occupied i, list = singles(i)
//   doubles : one group per alpha spin-orbital row i (warp chunks of 32 candidates if needed);
//             the candidates j > i of a row are the spin orbitals whose spatial index lies within
//             the band of non-empty pair lists (same spin: q in (p, p+B]; alpha rows also
//             opposite spin q in [p-B, p+B]), so a row fits one warp for local orbitals.  Beta
//             rows have only the B same-spin candidates; floor(32 / B) of them share a group.
// A warp takes one group; its active units (i and j occupied, list non-empty) are walked in
// order with the lanes over each unit's list entries.  Each group's CTMC rates are summed as
// exact 128-bit fixed-point integers (order independent) and stored; the CTMC kernel re-walks
// only the chosen group.  Every product that enters a rate uses explicitly rounded intrinsics
// so the two kernels compute bit-identical rates.
#include <math.h>

#include <algorithm>
#include <string>
#include <vector>

#include "common.cuh"

namespace {

__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float rsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double rexp(double x) { return exp(x); }
__device__ __forceinline__ float rexp(float x) { return expf(x); }
__device__ __forceinline__ double rrcp(double x) { return __ddiv_rn(1.0, x); }
__device__ __forceinline__ float rrcp(float x) { return __fdiv_rn(1.0f, x); }

// 16-byte vectors of the table precision, and f += sgn * x on them
template <typename real> struct Vec16;
template <> struct Vec16<float> { typedef float4 type; static constexpr int n = 4; };
template <> struct Vec16<double> { typedef double2 type; static constexpr int n = 2; };
__device__ __forceinline__ void vadd(float4 &f, float s, const float4 &x) {
    f.x += s * x.x; f.y += s * x.y; f.z += s * x.z; f.w += s * x.w;
}
__device__ __forceinline__ void vadd(double2 &f, double s, const double2 &x) { f.x += s * x.x; f.y += s * x.y; }
__device__ __forceinline__ float4 vfma2(float4 o, float x, float4 u, float y, float4 v) {   // o - x u - y v
    o.x = o.x - x * u.x - y * v.x; o.y = o.y - x * u.y - y * v.y;
    o.z = o.z - x * u.z - y * v.z; o.w = o.w - x * u.w - y * v.w;
    return o;
}
__device__ __forceinline__ double2 vfma2(double2 o, double x, double2 u, double y, double2 v) {
    o.x = o.x - x * u.x - y * v.x; o.y = o.y - x * u.y - y * v.y;
    return o;
}
// Fock-sum table (same-spin Tjk: 1, other-spin Tj: 0) in the table precision
template <typename real> __device__ __forceinline__ const real *fock_table(const ListsView &L, int same);
template <> __device__ __forceinline__ const float *fock_table<float>(const ListsView &L, int same) {
    return same ? L.Tjkf : L.Tjf;
}
template <> __device__ __forceinline__ const double *fock_table<double>(const ListsView &L, int same) {
    return same ? L.Tjk : L.Tj;
}

// One packed list record (16 B in the mixed form, 32 B in the FP64 form): key (a or a|b<<16)
// and up to three reals.
template <typename real> struct Rec;
template <> struct Rec<float> {
    float4 v;
    __device__ uint32_t key() const { return __float_as_uint(v.x); }
    __device__ float f1() const { return v.y; }
    __device__ float f2() const { return v.z; }
    __device__ float f3() const { return v.w; }
};
template <> struct Rec<double> {
    double4_32a v;
    __device__ uint32_t key() const { return (uint32_t)__double_as_longlong(v.x); }
    __device__ double f1() const { return v.y; }
    __device__ double f2() const { return v.z; }
    __device__ double f3() const { return v.w; }
};
__device__ __forceinline__ Rec<float> rec_single(const ListsView &L, uint32_t e, float) { return Rec<float>{__ldg(&L.s_rec32[e])}; }
__device__ __forceinline__ Rec<double> rec_single(const ListsView &L, uint32_t e, double) { return Rec<double>{L.s_rec64[e]}; }
__device__ __forceinline__ Rec<float> rec_same(const ListsView &L, uint32_t e, float) { return Rec<float>{__ldg(&L.ds_rec32[e])}; }
__device__ __forceinline__ Rec<double> rec_same(const ListsView &L, uint32_t e, double) { return Rec<double>{L.ds_rec64[e]}; }
__device__ __forceinline__ Rec<float> rec_opp(const ListsView &L, uint32_t e, float) { return Rec<float>{__ldg(&L.do_rec32[e])}; }
__device__ __forceinline__ Rec<double> rec_opp(const ListsView &L, uint32_t e, double) { return Rec<double>{L.do_rec64[e]}; }

// Walker arrays (global) and geometry.
struct WalkerArgs {
    int W, M, na, nb;
    const uint32_t *occ_bits;
    uint16_t *occ_list, *virt_list, *pos;
    uint32_t *occ_bits_w;
    void *G, *AinvT, *S, *F;
    double *e_diag;
    uint64_t *rng;
    uint16_t *cps;       // [W][n_corr] correlator indices (correlator product only)
};

struct SysDesc {
    ListsView L;
    WalkerArgs A;
    const double *J;
    double *e_loc, *t_res;
    u128 *rates;
    uint64_t *move_code;
    int w_begin;
};

struct Geo {
    int M, na, nb, ne, nw, nv_a, nv_b;
    size_t g_stride, a_stride;   // per-walker element strides of G and AinvT
    __device__ int n(int s) const { return s ? nb : na; }
    __device__ size_t g_off(int s) const { return s ? (size_t)nv_a * na : 0; }
    __device__ size_t a_off(int s) const { return s ? (size_t)na * na : 0; }
};

__device__ __forceinline__ Geo make_geo(int M, int na, int nb) {
    Geo g;
    g.M = M; g.na = na; g.nb = nb; g.ne = na + nb; g.nw = (M + 31) / 32;
    g.nv_a = M - na; g.nv_b = M - nb;
    g.g_stride = (size_t)(M - na) * na + (size_t)(M - nb) * nb;
    g.a_stride = (size_t)na * na + (size_t)nb * nb;
    return g;
}

// A work unit: one occupied spin orbital (single) or one occupied pair (double).
template <typename real>
struct Unit {
    uint32_t base, len;
    int kind;      // 0 single, 1 same-spin double, 2 opposite-spin double
    int cls;       // spin for kinds 0 and 1
    int ci, cj;    // columns of i and j
    int i, j;      // spin orbitals
    uint32_t sent; // key naming the unit's own (occupied) orbitals
    real einv;     // (1/E_i)(1/E_j)   (1/E_i for singles)
};

// Shared-memory view of one walker used by the entry evaluation.
template <typename real>
struct View {
    const uint16_t *pos;   // [2M]: occupied -> column, virtual -> 0x8000 | slot
    const real *Ga, *Gb;   // virtual rows of G per spin (shared and padded, or global)
    int lda, ldb;          // their row strides
    __device__ const real *Grow(int s, int slot) const {
        return s ? Gb + (size_t)slot * ldb : Ga + (size_t)slot * lda;
    }
    const real *E;         // [2M] exp(S_p) for virtual p, 1/exp(S_p) for occupied p (nullptr: compute
                           // from S on the fly)
    const real *S;         // walker S in global (used when E == nullptr)
    const real *F;         // walker F [2][ns_pad]
    CpsView C;             // correlator product (C.n_corr == 0: none)
    // its tables, staged in shared memory by the local energy (global otherwise): per-site
    // correlator lists, coefficient offsets, and per correlator the position of the walker's
    // current coefficient (cur == nullptr: val_off[l] + cidx[l] from the global indices) and 1/c
    const int32_t *soff, *voff, *cur;
    const uint32_t *sent;
    const uint16_t *cidx;  // [n_corr] the walker's correlator indices (global)
    const real *cinv;      // [n_corr] 1 / c_l[n_l] (shared), or nullptr: from the coefficients
    Geo geo;
    __device__ int cur_of(int l) const { return cur ? cur[l] : voff[l] + (int)cidx[l]; }
    __device__ real coef(int k) const;
    __device__ real cinv_of(int l) const { return cinv ? cinv[l] : rrcp(coef(cur_of(l))); }
    __device__ real Ev(int p) const { return E ? E[p] : rexp(S[p]); }              // p virtual
    __device__ real Eiv(int p) const { return E ? E[p] : rrcp(rexp(S[p])); }       // p occupied
    __device__ bool occ(int p) const { return !(pos[p] & 0x8000); }
};

// Correlator coefficient k in the table precision (the mixed form reads the FP32 copy).
template <> __device__ __forceinline__ float View<float>::coef(int k) const { return __ldg(&C.values32[k]); }
template <> __device__ __forceinline__ double View<double>::coef(int k) const { return __ldg(&C.values[k]); }

template <typename real> __device__ __forceinline__ real V0coef(const CpsView &C, int k);
template <> __device__ __forceinline__ float V0coef<float>(const CpsView &C, int k) { return C.values32[k]; }
template <> __device__ __forceinline__ double V0coef<double>(const CpsView &C, int k) { return C.values[k]; }

// Point a view's correlator tables at the global copies (the CTMC choice, the move set).
template <typename real>
__device__ __forceinline__ void cps_global(View<real> &V, const CpsView &C, const uint16_t *cidx) {
    V.C = C; V.soff = C.site_off; V.sent = C.site_ent; V.voff = C.val_off; V.cur = nullptr;
    V.cidx = cidx; V.cinv = nullptr;
}

// Correlator-product ratio prod_l c_l[n_l + delta_l] / c_l[n_l] of the move that empties spin
// orbitals r0 (and r1) and fills a0 (and a1) (Sec. III.B): the per-site lists of the changed sites
// are merged in correlator order so every touched correlator is visited once, with delta_l the sum
// of the digit changes (+-1 alpha, +-2 beta) times 4^(site position).  nx = 2 (single) or 4.
// A state index outside the correlator's table (an inconsistent state) gives NaN, which the rate
// check reports.
template <typename real>
__device__ __forceinline__ real cps_ratio(const View<real> &V, int r0, int a0, int r1, int a1, int nx) {
    const int M = V.geo.M;
    int h[4], e[4], d[4];
    uint32_t c[4];
#pragma unroll
    for (int x = 0; x < 4; ++x) {
        const int p = x == 0 ? r0 : (x == 1 ? a0 : (x == 2 ? r1 : a1));
        const int sp = p >= M ? 1 : 0, site = p - sp * M;
        d[x] = ((x & 1) ? 1 : -1) * (1 + sp);
        h[x] = x < nx ? V.soff[site] : 0;
        e[x] = x < nx ? V.soff[site + 1] : 0;
        c[x] = h[x] < e[x] ? V.sent[h[x]] : 0xFFFFFFFFu;
    }
    real r = real(1);
    for (int it = 0; it < 4 * VMC_CPS_MAX_PER_SITE; ++it) {
        const uint32_t l = min(min(c[0], c[1]), min(c[2], c[3])) >> 16;   // next correlator, ascending
        if (l == 0xFFFFu) break;
        int delta = 0;
#pragma unroll
        for (int x = 0; x < 4; ++x)
            if ((c[x] >> 16) == l) {
                delta += d[x] * (int)(c[x] & 0xFFFFu);
                ++h[x];
                c[x] = h[x] < e[x] ? V.sent[h[x]] : 0xFFFFFFFFu;
            }
        const int k = V.cur_of((int)l) + delta;
        if (k < V.voff[l] || k >= V.voff[l + 1]) return real(NAN);
        r = rmul(r, rmul(V.coef(k), V.cinv_of((int)l)));
    }
    return r;
}

// Unit of lane `lane` in group g, from the lists' unit table (the static (group, lane) -> (i, j,
// list) map, with the list lengths of the current eps_run): active if the list is non-empty and i
// (and j) are occupied in this walker.  Returns false if the lane has no active unit.
template <typename real>
__device__ __forceinline__ bool setup_unit(const ListsView &L, const View<real> &V, int g, int lane,
                                           Unit<real> &u) {
    const int M = L.M;
    const uint4 t = __ldg(&L.unit_tab[(size_t)g * 32 + lane]);
    u.base = t.y; u.len = t.z; u.kind = (int)(t.w & 3); u.cls = (int)(t.w >> 2); u.sent = t.x;
    u.ci = 0; u.cj = 0; u.einv = real(0);
    const int lo = (int)(t.x & 0xFFFFu), hi = (int)(t.x >> 16);
    u.i = u.kind == 2 ? lo : u.cls * M + lo;
    u.j = u.kind == 0 ? -1 : (u.kind == 2 ? M + hi : u.cls * M + hi);
    if (u.len == 0 || !V.occ(u.i)) return false;
    if (u.kind != 0 && !V.occ(u.j)) return false;
    u.ci = V.pos[u.i];
    if (u.kind == 0) {
        u.einv = V.Eiv(u.i);
    } else {
        u.cj = V.pos[u.j];
        u.einv = rmul(V.Eiv(u.i), V.Eiv(u.j));
    }
    return true;
}

template <typename real>
__device__ __forceinline__ Unit<real> shfl_unit(const Unit<real> &u, int src) {
    Unit<real> v;
    v.base = __shfl_sync(0xffffffffu, u.base, src);
    v.len = __shfl_sync(0xffffffffu, u.len, src);
    v.kind = __shfl_sync(0xffffffffu, u.kind, src);
    v.cls = __shfl_sync(0xffffffffu, u.cls, src);
    v.ci = __shfl_sync(0xffffffffu, u.ci, src);
    v.cj = __shfl_sync(0xffffffffu, u.cj, src);
    v.i = __shfl_sync(0xffffffffu, u.i, src);
    v.j = __shfl_sync(0xffffffffu, u.j, src);
    v.einv = __shfl_sync(0xffffffffu, u.einv, src);
    return v;
}

// Are the target orbital(s) of entry idx unoccupied?  Reads only the 2- or 4-byte key.
template <typename real>
__device__ __forceinline__ bool entry_free(const ListsView &L, const View<real> &V, int kind, int cls,
                                           uint32_t idx) {
    const int M = V.geo.M;
    if (kind == 0) return V.pos[cls * M + __ldg(&L.s_a[idx])] & 0x8000;
    if (kind == 1) {
        const uint32_t ab = __ldg(&L.ds_ab[idx]);
        return V.pos[cls * M + (ab & 0xFFFF)] & V.pos[cls * M + (ab >> 16)] & 0x8000;
    }
    const uint32_t ab = __ldg(&L.do_ab[idx]);
    return V.pos[ab & 0xFFFF] & V.pos[M + (ab >> 16)] & 0x8000;
}

__device__ __forceinline__ uint32_t list_size(const ListsView &L, int kind) {
    return (uint32_t)(kind == 0 ? L.ns : (kind == 1 ? L.nds : L.ndo));
}

// ratio = psi(m)/psi(n) of a free entry (in-place replacement convention: the fermionic phases
// of H and of the ratio cancel) and contrib = H_nm * ratio.  Every kernel evaluates rates with
// this one sequence of explicitly rounded operations, so they agree bit for bit.
template <typename real, bool kC>
__device__ __forceinline__ void entry_value(const ListsView &L, const View<real> &V, int kind, int cls, int ci,
                                            int cj, real einv, uint32_t idx, real &ratio, real &contrib, int &A,
                                            int &B, int I = -1, int Jo = -1) {
    const int M = V.geo.M;
    if (kind == 0) {
        const int s = cls;
        const Rec<real> r = rec_single(L, idx, real(0));
        const int a = (int)r.key();
        const real g = V.Grow(s, V.pos[s * M + a] & 0x7FFF)[ci];
        const real w = s ? r.f2() : r.f1();
        real rt = rmul(rmul(rmul(g, w), V.Ev(s * M + a)), einv);
        if (kC) rt = rmul(rt, cps_ratio<real>(V, I, s * M + a, I, s * M + a, 2));
        ratio = rt;
        contrib = rmul(V.F[(size_t)s * L.ns_pad + idx], rt);
        A = s * M + a; B = -1;
        return;
    }
    if (kind == 1) {
        const int s = cls;
        const Rec<real> r = rec_same(L, idx, real(0));
        const uint32_t ab = r.key();
        const int a = ab & 0xFFFF, b = ab >> 16;
        const real *ra = V.Grow(s, V.pos[s * M + a] & 0x7FFF);
        const real *rb = V.Grow(s, V.pos[s * M + b] & 0x7FFF);
        const real minor = rsub(rmul(ra[ci], rb[cj]), rmul(ra[cj], rb[ci]));
        const real w = s ? r.f3() : r.f2();
        real rt = rmul(rmul(rmul(rmul(minor, w), V.Ev(s * M + a)), V.Ev(s * M + b)), einv);
        if (kC) rt = rmul(rt, cps_ratio<real>(V, I, s * M + a, Jo, s * M + b, 4));
        ratio = rt;
        contrib = rmul(r.f1(), rt);
        A = s * M + a; B = s * M + b;
        return;
    }
    const Rec<real> r = rec_opp(L, idx, real(0));
    const uint32_t ab = r.key();
    const int a = ab & 0xFFFF, b = ab >> 16;
    const real ga = V.Grow(0, V.pos[a] & 0x7FFF)[ci];
    const real gb = V.Grow(1, V.pos[M + b] & 0x7FFF)[cj];
    real rt = rmul(rmul(rmul(rmul(rmul(ga, gb), r.f2()), V.Ev(a)), V.Ev(M + b)), einv);
    if (kC) rt = rmul(rt, cps_ratio<real>(V, I, a, Jo, M + b, 4));
    ratio = rt;
    contrib = rmul(r.f1(), rt);
    A = a; B = M + b;
}

// Evaluate list entry `idx` of unit u.  Returns false if the target orbital(s) are occupied.
template <typename real, bool kC>
__device__ __forceinline__ bool eval_entry(const ListsView &L, const View<real> &V, const Unit<real> &u,
                                           uint32_t idx, real &ratio, real &contrib, int &A, int &B) {
    if (!entry_free<real>(L, V, u.kind, u.cls, idx)) return false;
    entry_value<real, kC>(L, V, u.kind, u.cls, u.ci, u.cj, u.einv, idx, ratio, contrib, A, B, u.i, u.j);
    return true;
}

template <typename real>
__device__ __forceinline__ u128 rate_of(real ratio, unsigned *flag) {
    real r = fabs(ratio);
    if (!(r < (real)8796093022208.0)) {   // 2^43: fixed-point range limit (also catches NaN)
        *flag |= VMC_DEV_OVERFLOW;
        r = (r == r) ? (real)8796093022207.0 : (real)0;
    }
    return rate_fixed(r);
}

template <typename real> struct AccT { typedef double type; };
template <> struct AccT<float> { typedef float type; };

__device__ __forceinline__ double warp_sum_acc(double v) { return warp_sum_f64(v); }
__device__ __forceinline__ double warp_sum_acc(float v) {
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
    return (double)v;
}

// Evaluate cnt queued entries q[0..cnt) of one warp, one per lane (lanes >= cnt idle).  Every entry
// of one queue has the same kind K (compile time).  Entry code = list index << 5 | unit lane; the
// unit's columns, 1/(E_i E_j) and kind | spin << 2 are held by that lane (cci, ccj, ceinv, cmeta).
template <int K, typename real, typename acc_t, bool kC>
__device__ __forceinline__ void drain_queue(const ListsView &L, const View<real> &V, const uint32_t *q, int cnt,
                                            int lane, int cci, int ccj, real ceinv, int cmeta, int cii, int cjj,
                                            acc_t &e_grp, u128 &q_grp, unsigned &flag) {
    const uint32_t code = lane < cnt ? q[lane] : 0u;
    const int src = (int)(code & 31u);
    const int ci = __shfl_sync(0xffffffffu, cci, src);
    const int cj = K == 0 ? 0 : __shfl_sync(0xffffffffu, ccj, src);
    const real einv = __shfl_sync(0xffffffffu, ceinv, src);
    const int cls = K == 2 ? 0 : (__shfl_sync(0xffffffffu, cmeta, src) >> 2);
    const int oi = kC ? __shfl_sync(0xffffffffu, cii, src) : -1;
    const int oj = (kC && K != 0) ? __shfl_sync(0xffffffffu, cjj, src) : -1;
    if (lane < cnt) {
        real ratio, contrib;
        int a, b;
        entry_value<real, kC>(L, V, K, cls, ci, cj, einv, code >> 5, ratio, contrib, a, b, oi, oj);
        e_grp += (acc_t)contrib;
        q_grp += rate_of<real>(ratio, &flag);
    }
}

// Packed walk over a range [f0, f1) of the concatenated lists of a group's active units, all of
// entry kind K (compile time).  The active units sit in lanes 0 .. n_act-1 in canonical order, with
// strictly increasing inclusive length prefix incl (the lanes after them hold incl = total).  Each
// pass reads 32 consecutive entries of the concatenation, one per lane: lane l takes flat entry
// f = c0 + l, whose unit is the number of units
// ending at or before f, counted as the units ending at or before c0 (a ballot) plus those ending
// inside the pass (one bit each, gathered by a warp OR-reduction, then a popcount below the lane).
// Each lane loads its entry's 2- or 4-byte key, tests the target orbital(s) in the shared orbital
// map and queues the free entries; every 32 queued entries are evaluated at once.  Entry code =
// list index << 5 | unit lane; a unit's list index of flat entry f is f + (list base - unit start),
// one shuffle.  Lanes past f1 read entry 0 of the list (always allocated) and queue nothing, so the
// test needs no bounds branch.  pos and the queues are 32-bit shared addresses.
template <int K, typename real, typename acc_t, bool kC>
__device__ __forceinline__ void walk_range(const ListsView &L, const View<real> &V, uint32_t f0, uint32_t f1,
                                           uint32_t incl, uint32_t cdelta, int cmeta, int cls_row,
                                           uint32_t *wq, int &qn, int lane, unsigned lt_mask,
                                           int cci, int ccj, real ceinv, int cii, int cjj, acc_t &e_grp, u128 &q_grp,
                                           unsigned &flag) {
    const int M = V.geo.M;
    const uint32_t sPos = (uint32_t)__cvta_generic_to_shared(V.pos);
    uint32_t *q = K == 2 ? wq + 64 : wq;
    const uint32_t sQ = (uint32_t)__cvta_generic_to_shared(q);
    const uint32_t low = lane == 31 ? 0xFFFFFFFEu : ((2u << lane) - 2u);   // bits 1 .. lane
    const uint32_t oA = K == 2 ? 0u : (uint32_t)(cls_row * M), oB = K == 2 ? (uint32_t)M : oA;
    for (uint32_t c0 = f0; c0 < f1; c0 += 32) {
        const uint32_t f = c0 + lane;
        // lanes past the active units hold incl = total > c0, so they never count as "before";
        // a unit ending at or before c0 has end = 0 (bit 0, never counted) or end >= 2^31 (no bit)
        const unsigned before = __ballot_sync(0xffffffffu, incl <= c0);
        const uint32_t end = incl - c0;
        uint32_t bit;
        asm("shl.b32 %0, 1, %1;" : "=r"(bit) : "r"(end));   // PTX clamps shifts >= 32: no bit
        const uint32_t inside = __reduce_or_sync(0xffffffffu, bit);
        // for valid lanes su < n_act; past f1 it may be 32, which the shuffles take modulo 32
        const int su = __popc(before) + __popc(inside & low);
        const bool valid = f < f1;
        const uint32_t idx = __shfl_sync(0xffffffffu, cdelta, su) + f;   // list base - unit start + f
        const uint32_t ridx = valid ? idx : 0u;
        uint32_t x, y = 0xFFFFu;
        if (K == 0) {
            const int cls = __shfl_sync(0xffffffffu, cmeta, su) >> 2;
            const uint32_t key = (uint32_t)__ldg(&L.s_a[ridx]);
            asm("ld.shared.u16 %0, [%1];" : "=r"(x) : "r"(sPos + 2u * ((uint32_t)(cls * M) + (key & 0xFFFFu))));
        } else {
            const uint32_t key = __ldg((K == 2 ? L.do_ab : L.ds_ab) + ridx);
            asm("ld.shared.u16 %0, [%1];" : "=r"(x) : "r"(sPos + 2u * (oA + (key & 0xFFFFu))));
            asm("ld.shared.u16 %0, [%1];" : "=r"(y) : "r"(sPos + 2u * (oB + (key >> 16))));
        }
        const bool pass = valid && (x & y & 0x8000u);
        const unsigned bal = __ballot_sync(0xffffffffu, pass);
        if (pass)
            asm volatile("st.shared.u32 [%0], %1;" ::"r"(sQ + 4u * (uint32_t)(qn + __popc(bal & lt_mask))),
                         "r"((idx << 5) | (uint32_t)su) : "memory");
        qn += __popc(bal);
        if (qn >= 32) {
            __syncwarp();
            qn -= 32;
            drain_queue<K, real, acc_t, kC>(L, V, q + qn, 32, lane, cci, ccj, ceinv, cmeta, cii, cjj, e_grp, q_grp,
                                            flag);
            __syncwarp();
        }
    }
}

// Local energy of walker w by the whole CTA (any number of warps).  smraw: dynamic shared memory.
template <typename real, bool kC>
__device__ __forceinline__ void eloc_walker(const ListsView &L, const WalkerArgs &A, const int w,
                                            double *__restrict__ e_loc, double *__restrict__ t_res,
                                            u128 *__restrict__ rates, unsigned *status, unsigned char *smraw,
                                            const CpsView &C = CpsView{}) {
    const Geo geo = make_geo(A.M, A.na, A.nb);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nt = blockDim.x, nwarp = nt >> 5;
    const int M = geo.M, n_groups = L.n_groups, n_sgl_groups = (2 * M + 31) / 32;
    const int lda = geo.na + 1, ldb = geo.nb + 1;    // padded rows: no bank conflicts on columns
    real *sGa = (real *)smraw;
    real *sGb = sGa + (size_t)geo.nv_a * lda;
    real *sE = sGb + (size_t)geo.nv_b * ldb;
    uint16_t *pos = (uint16_t *)(sE + 2 * M);
    // per-group energy partials: global, after the system's rate sums (written and read by this CTA)
    double *eg = (double *)(rates + (size_t)A.W * n_groups) + (size_t)w * n_groups;
    // per warp: two queues of 64 entry codes (idx << 5 | unit lane): kinds 0/1, and kind 2
    uint32_t *wq = (uint32_t *)(((uintptr_t)(pos + 2 * M) + 15) & ~(uintptr_t)15) + warp * 128;
    // correlator product, after the queues: 1 / c_l[n_l], the current coefficient positions, the
    // coefficient offsets and the per-site correlator lists
    real *sCinv = (real *)((uint32_t *)(((uintptr_t)(pos + 2 * M) + 15) & ~(uintptr_t)15) + nwarp * 128);
    int32_t *sCur = (int32_t *)(sCinv + ((C.n_corr + 3) & ~3));
    int32_t *sVoff = sCur + C.n_corr;
    int32_t *sSoff = sVoff + C.n_corr + 1;
    uint32_t *sSent = (uint32_t *)(sSoff + M + 1);
    __shared__ u128 red_q[32];
    __shared__ int next_group;

    // ---- prologue: stage G into padded rows, exp(S), orbital map
    {
        const real *Gw = (const real *)A.G + (size_t)w * geo.g_stride;
        const size_t na_el = (size_t)geo.nv_a * geo.na;
        for (int r = warp; r < geo.nv_a + geo.nv_b; r += nwarp) {   // one row per warp
            const bool bs = r >= geo.nv_a;
            const int rr = bs ? r - geo.nv_a : r, n = bs ? geo.nb : geo.na;
            const real *src = Gw + (bs ? na_el + (size_t)rr * geo.nb : (size_t)rr * geo.na);
            real *dst = bs ? sGb + (size_t)rr * ldb : sGa + (size_t)rr * lda;
            for (int c = lane; c < n; c += 32) dst[c] = src[c];
        }
        const real *Sw = (const real *)A.S + (size_t)w * 2 * M;
        const uint16_t *pw = A.pos + (size_t)w * 2 * M;
        for (int p = tid; p < 2 * M; p += nt) {
            const uint16_t ps = pw[p];
            const real e = rexp(Sw[p]);
            sE[p] = (ps & 0x8000) ? e : rrcp(e);
            pos[p] = ps;
        }
        if (kC) {
            for (int l = tid; l <= C.n_corr; l += nt) sVoff[l] = C.val_off[l];
            for (int k = tid; k <= M; k += nt) sSoff[k] = C.site_off[k];
            for (int k = tid; k < C.nnz; k += nt) sSent[k] = C.site_ent[k];
            for (int l = tid; l < C.n_corr; l += nt) {
                const int k = C.val_off[l] + (int)A.cps[(size_t)w * C.n_corr + l];
                sCur[l] = k;
                sCinv[l] = rrcp(V0coef<real>(C, k));
            }
        }
        if (tid == 0) next_group = nwarp;
    }
    __syncthreads();

    View<real> V;
    V.pos = pos; V.Ga = sGa; V.Gb = sGb; V.lda = lda; V.ldb = ldb;
    V.E = sE; V.S = nullptr; V.F = (const real *)A.F + (size_t)w * 2 * L.ns_pad; V.geo = geo;
    V.C = C; V.soff = sSoff; V.sent = sSent; V.voff = sVoff; V.cur = sCur; V.cidx = nullptr; V.cinv = sCinv;
    typedef typename AccT<real>::type acc_t;
    u128 q_tot = 0;
    unsigned flag = 0;

    // Groups are taken dynamically; each group's sums are stored by index, so the result does not
    // depend on which warp took it.  Inside a group the warp walks the units' lists with a cheap
    // key check and queues the entries whose targets are free; the ratio, rate and energy of
    // queued entries are evaluated 32 at a time, one per lane, so that work is never divergent.
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int g = warp; g < n_groups;) {
        Unit<real> u;
        const bool act = setup_unit<real>(L, V, g, lane, u);
        acc_t e_grp = 0;
        u128 q_grp = 0;
        unsigned amask = __ballot_sync(0xffffffffu, act);
        if (__ballot_sync(0xffffffffu, act && u.base + u.len > list_size(L, u.kind))) {   // cannot happen: guard
            flag |= VMC_DEV_INCONSISTENT;
            amask = 0;
        }
        const int n_act = __popc(amask);
        if (n_act == 0) {                // an empty group (its row orbital unoccupied): zero sums
            if (lane == 0) {
                rates[(size_t)w * n_groups + g] = 0;
                eg[g] = 0.0;
            }
            int nxt = 0;
            if (lane == 0) nxt = atomicAdd(&next_group, 1);
            g = __shfl_sync(0xffffffffu, nxt, 0);
            continue;
        }
        // compact the active units into lanes 0 .. n_act-1, in order (same-spin units precede the
        // opposite-spin ones of a row); the queue, empty between groups, holds the permutation
        const int n1 = __popc(amask & __ballot_sync(0xffffffffu, u.kind != 2));
        if ((amask >> lane) & 1u) wq[__popc(amask & lt_mask)] = (uint32_t)lane;
        __syncwarp();
        const int src = lane < n_act ? (int)wq[lane] : lane;
        __syncwarp();
        const uint32_t clen0 = __shfl_sync(0xffffffffu, u.len, src);
        const uint32_t clen = lane < n_act ? clen0 : 0u;
        const uint32_t cbase = __shfl_sync(0xffffffffu, u.base, src);
        const int cmeta = __shfl_sync(0xffffffffu, u.kind | (u.cls << 2), src);
        const int cci = __shfl_sync(0xffffffffu, u.ci, src), ccj = __shfl_sync(0xffffffffu, u.cj, src);
        const int cii = kC ? __shfl_sync(0xffffffffu, u.i, src) : 0, cjj = kC ? __shfl_sync(0xffffffffu, u.j, src) : 0;
        const real ceinv = __shfl_sync(0xffffffffu, u.einv, src);
        // inclusive prefix of the compacted list lengths; t1 = end of the same-spin (or singles) part
        uint32_t incl = clen;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t o = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += o;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        const uint32_t cdelta = cbase - (incl - clen);   // list index of flat entry f: f + cdelta (mod 2^32)
        const uint32_t t1v = __shfl_sync(0xffffffffu, incl, n1 > 0 ? n1 - 1 : 0), t1 = n1 > 0 ? t1v : 0u;
        const int cls_row = __shfl_sync(0xffffffffu, cmeta, 0) >> 2;   // spin of a row group's same-spin units
        int qn0 = 0, qn1 = 0;   // queue fill (warp-uniform)
        if (g < n_sgl_groups) {
            walk_range<0, real, acc_t, kC>(L, V, 0, total, incl, cdelta, cmeta, 0, wq, qn0, lane, lt_mask,
                                           cci, ccj, ceinv, cii, cjj, e_grp, q_grp, flag);
            __syncwarp();
            if (qn0)
                drain_queue<0, real, acc_t, kC>(L, V, wq, qn0, lane, cci, ccj, ceinv, cmeta, cii, cjj, e_grp, q_grp,
                                                flag);
        } else {
            walk_range<1, real, acc_t, kC>(L, V, 0, t1, incl, cdelta, cmeta, cls_row, wq, qn0, lane, lt_mask,
                                           cci, ccj, ceinv, cii, cjj, e_grp, q_grp, flag);
            walk_range<2, real, acc_t, kC>(L, V, t1, total, incl, cdelta, cmeta, cls_row, wq, qn1, lane,
                                           lt_mask, cci, ccj, ceinv, cii, cjj, e_grp, q_grp, flag);
            __syncwarp();
            if (qn0)
                drain_queue<1, real, acc_t, kC>(L, V, wq, qn0, lane, cci, ccj, ceinv, cmeta, cii, cjj, e_grp, q_grp,
                                                flag);
            if (qn1)
                drain_queue<2, real, acc_t, kC>(L, V, wq + 64, qn1, lane, cci, ccj, ceinv, cmeta, cii, cjj, e_grp,
                                                q_grp, flag);
        }
        __syncwarp();
        const double eg_sum = warp_sum_acc(e_grp);   // FP32 lanes in the mixed form: one conversion
        q_grp = warp_sum_u128(q_grp);
        if (lane == 0) {
            rates[(size_t)w * n_groups + g] = q_grp;
            eg[g] = eg_sum;
        }
        q_tot += q_grp;
        int nxt = 0;
        if (lane == 0) nxt = atomicAdd(&next_group, 1);
        g = __shfl_sync(0xffffffffu, nxt, 0);
    }
    if (lane == 0) red_q[warp] = q_tot;
    if (flag) atomicOr(status, flag);
    __syncthreads();
    if (warp == 0) {
        // fixed-order sum of the per-group energies: lane l takes groups l, l+32, ...
        double s = 0.0;
        for (int g = lane; g < n_groups; g += 32) s += eg[g];
        s = warp_sum_f64(s);
        if (lane == 0) {
            u128 Q = 0;
            for (int k = 0; k < nwarp; ++k) Q += red_q[k];
            e_loc[w] = A.e_diag[w] + s;
            if (Q == 0) {
                t_res[w] = 0.0;
                atomicOr(status, VMC_DEV_NOMOVE);
            } else {
                const double qh = (double)(uint64_t)(Q >> 64), ql = (double)(uint64_t)Q;
                t_res[w] = __ddiv_rn(1.0, __dadd_rn(qh, __dmul_rn(ql, 0x1p-64)));
            }
        }
    }
    __syncthreads();   // shared memory may be reused for the next walker
}

// CTA widths the local-energy kernels are built for (128, 256, 384, 512 threads), each with the
// minimum of resident CTAs per SM that keeps it at <= 64 registers per thread, so that shared
// memory (the walker's G rows) rather than registers bounds the CTAs per SM.
template <int kT> struct EmB { static constexpr int v = kT >= 512 ? 2 : (kT >= 384 ? 3 : (kT >= 256 ? 4 : 8)); };

template <typename real, int kT>
__global__ void __launch_bounds__(kT, EmB<kT>::v)
k_local_energy(ListsView L, WalkerArgs A, double *__restrict__ e_loc, double *__restrict__ t_res,
               u128 *__restrict__ rates, unsigned *status) {
    extern __shared__ __align__(16) unsigned char smraw[];
    eloc_walker<real, false>(L, A, blockIdx.x, e_loc, t_res, rates, status, smraw);
}

// The same with the correlator product (a separate instantiation, so the pair-Jastrow kernel above
// is not touched by it).
template <typename real, int kT>
__global__ void __launch_bounds__(kT, EmB<kT>::v)
k_local_energy_cps(ListsView L, WalkerArgs A, CpsView C, double *__restrict__ e_loc, double *__restrict__ t_res,
                   u128 *__restrict__ rates, unsigned *status) {
    extern __shared__ __align__(16) unsigned char smraw[];
    eloc_walker<real, true>(L, A, blockIdx.x, e_loc, t_res, rates, status, smraw, C);
}

// Batched launch over several systems (uneven sizes).  CTAs stay resident and take walkers from
// a global queue; the descriptors are ordered by decreasing cost so the long walkers start first.
template <typename real, int kT>
__global__ void __launch_bounds__(kT, EmB<kT>::v)
k_local_energy_batched(const SysDesc *__restrict__ sys, int n_sys, int total, int *queue, unsigned *status) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(queue, 1);
        __syncthreads();
        const int t = s_item;
        __syncthreads();
        if (t >= total) break;
        int k = 0;
        while (k + 1 < n_sys && sys[k + 1].w_begin <= t) ++k;
        const SysDesc &d = sys[k];
        eloc_walker<real, false>(d.L, d.A, t - d.w_begin, d.e_loc, d.t_res, d.rates, status, smraw);
    }
}

// ---------------------------------------------------------------------------------- CTMC
// Selection: one warp per walker.  Scans the walker's group sums (u128), draws Philox, finds the
// group whose prefix crosses T and re-walks only that group with the same entry code as the
// local-energy kernel.  Writes the move code (0 = no move) and advances the walker's counter.
template <typename real, bool kC>
__device__ __forceinline__ void select_walker(const ListsView &L, const WalkerArgs &A, const int w,
                                              const u128 *__restrict__ rates, uint64_t seed,
                                              uint64_t *__restrict__ move_code, unsigned *status,
                                              const CpsView &C = CpsView{}) {
    const Geo geo = make_geo(A.M, A.na, A.nb);
    const int lane = threadIdx.x & 31;
    const int M = geo.M, N2 = 2 * M, n_groups = L.n_groups;
    const real *Gw = (const real *)A.G + (size_t)w * geo.g_stride;
    const real *Sw = (const real *)A.S + (size_t)w * N2;
    const u128 *R = rates + (size_t)w * n_groups;
    const int per = (n_groups + 31) / 32;
    const int g0 = lane * per, g1 = min(n_groups, g0 + per);
    u128 seg = 0;
    for (int g = g0; g < g1; ++g) seg += R[g];
    const u128 incl = warp_incl_scan_u128(seg, lane);
    const u128 Q = shfl_u128(incl, 31);
    const uint64_t U = philox4x64_word0(A.rng[w], 0, 0, 0, seed, (uint64_t)w);
    const uint64_t qh = (uint64_t)(Q >> 64), ql = (uint64_t)Q;
    const u128 T = (u128)U * qh + (u128)__umul64hi(U, ql);
    const unsigned ball = __ballot_sync(0xffffffffu, incl > T);
    int gsel = -1;
    u128 before = 0;
    if (Q != 0 && ball) {
        const int src = __ffs(ball) - 1;
        u128 pre = shfl_u128(incl - seg, src);
        if (lane == src) {
            for (int g = g0; g < g1; ++g) {
                if (pre + R[g] > T) { gsel = g; break; }
                pre += R[g];
            }
        }
        gsel = __shfl_sync(0xffffffffu, gsel, src);
        before = shfl_u128(pre, src);
    }
    uint64_t code = 0;
    if (gsel >= 0) {
        const u128 Tl = T - before;   // threshold inside the group
        View<real> V;
        V.pos = A.pos + (size_t)w * N2; V.Ga = Gw; V.Gb = Gw + geo.g_off(1); V.lda = geo.na; V.ldb = geo.nb;
        V.E = nullptr; V.S = Sw; V.F = (const real *)A.F + (size_t)w * 2 * L.ns_pad; V.geo = geo;
        if (kC) cps_global(V, C, A.cps + (size_t)w * C.n_corr);
        Unit<real> u;
        const bool act = setup_unit<real>(L, V, gsel, lane, u);
        unsigned mask = __ballot_sync(0xffffffffu, act);
        u128 carry = 0;
        unsigned flag = 0;
        bool found = false;
        while (mask && !found) {
            const int src = __ffs(mask) - 1;
            mask &= mask - 1;
            const Unit<real> v = shfl_unit(u, src);
            for (uint32_t k0 = 0; k0 < v.len && !found; k0 += 32) {
                const uint32_t k = k0 + lane;
                u128 q = 0;
                int a = -1, b = -1;
                if (k < v.len) {
                    real ratio, contrib;
                    if (eval_entry<real, kC>(L, V, v, v.base + k, ratio, contrib, a, b)) q = rate_of<real>(ratio, &flag);
                }
                const u128 incl2 = warp_incl_scan_u128(q, lane) + carry;
                const unsigned hit = __ballot_sync(0xffffffffu, k < v.len && q != 0 && incl2 > Tl);
                if (hit) {
                    const int h = __ffs(hit) - 1;
                    uint64_t c = 0;
                    if (lane == h) {
                        const uint64_t kind = v.kind == 0 ? 1 : 2;
                        const uint64_t j10 = kind == 2 ? (uint64_t)v.j : 1023ull, b10 = kind == 2 ? (uint64_t)b : 1023ull;
                        c = kind | ((uint64_t)v.i << 2) | (j10 << 12) | ((uint64_t)a << 22) | (b10 << 32);
                    }
                    code = __shfl_sync(0xffffffffu, c, h);
                    found = true;
                }
                carry = shfl_u128(incl2, 31);
            }
        }
        if (!found && lane == 0) atomicOr(status, VMC_DEV_INCONSISTENT);
    } else if (lane == 0) {
        atomicOr(status, VMC_DEV_NOMOVE);
    }
    if (lane == 0) {
        move_code[w] = code;
        A.rng[w] += 1;
    }
}

template <typename real, bool kC>
__global__ void __launch_bounds__(512)
k_ctmc_select(ListsView L, WalkerArgs A, CpsView C, const u128 *__restrict__ rates, uint64_t seed,
              uint64_t *__restrict__ move_code, unsigned *status) {
    const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (w >= A.W) return;
    select_walker<real, kC>(L, A, w, rates, seed, move_code, status, C);
}

template <typename real>
__global__ void __launch_bounds__(512)
k_ctmc_select_batched(const SysDesc *__restrict__ sys, int n_sys, int total, uint64_t seed, unsigned *status) {
    const int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (t >= total) return;
    int k = 0;
    while (k + 1 < n_sys && sys[k + 1].w_begin <= t) ++k;
    const SysDesc &d = sys[k];
    select_walker<real, false>(d.L, d.A, t - d.w_begin, d.rates, seed, d.move_code, status);
}

// Screened move set of one walker, written out in canonical order (Sec. II.A, II.B): one warp per
// walker walks the same groups, units and list entries as the local energy (groups in index order,
// units in lane order, entries in list order) and writes every entry whose targets are free with
// the ratio and contribution the local energy and the CTMC choice use.  Diagnostic path: it also
// counts the list entries the walk reads (singles, doubles), free or not.
template <typename real, bool kC>
__global__ void __launch_bounds__(256)
k_screened_moves(ListsView L, WalkerArgs A, CpsView C, int w_begin, int n_w, int64_t cap, uint64_t *__restrict__ code_out,
                 double *__restrict__ ratio_out, double *__restrict__ contrib_out, int64_t *__restrict__ count_out,
                 int64_t *__restrict__ walked_out, unsigned *status) {
    const int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (t >= n_w) return;
    const int w = w_begin + t;
    const int lane = threadIdx.x & 31;
    const Geo geo = make_geo(A.M, A.na, A.nb);
    const int M = geo.M, N2 = 2 * M;
    const real *Gw = (const real *)A.G + (size_t)w * geo.g_stride;
    View<real> V;
    V.pos = A.pos + (size_t)w * N2; V.Ga = Gw; V.Gb = Gw + geo.g_off(1); V.lda = geo.na; V.ldb = geo.nb;
    V.E = nullptr; V.S = (const real *)A.S + (size_t)w * N2; V.F = (const real *)A.F + (size_t)w * 2 * L.ns_pad;
    V.geo = geo;
    if (kC) cps_global(V, C, A.cps + (size_t)w * C.n_corr);
    const unsigned lt_mask = (1u << lane) - 1u;
    int64_t cnt = 0, walked_s = 0, walked_d = 0;
    unsigned flag = 0;
    for (int g = 0; g < L.n_groups; ++g) {
        Unit<real> u;
        const bool act = setup_unit<real>(L, V, g, lane, u);
        unsigned mask = __ballot_sync(0xffffffffu, act);
        while (mask) {
            const int src = __ffs(mask) - 1;
            mask &= mask - 1;
            const Unit<real> v = shfl_unit(u, src);
            if (v.base + v.len > list_size(L, v.kind)) {   // cannot happen: guard, never read
                flag |= VMC_DEV_INCONSISTENT;
                continue;
            }
            if (v.kind == 0) walked_s += v.len; else walked_d += v.len;
            for (uint32_t k0 = 0; k0 < v.len; k0 += 32) {
                const uint32_t k = k0 + lane;
                real ratio = 0, contrib = 0;
                int a = -1, b = -1;
                const bool fr = k < v.len && eval_entry<real, kC>(L, V, v, v.base + k, ratio, contrib, a, b);
                const unsigned bal = __ballot_sync(0xffffffffu, fr);
                if (fr) {
                    const int64_t p = cnt + __popc(bal & lt_mask);
                    if (p < cap) {
                        const uint64_t kind = v.kind == 0 ? 1 : 2;
                        const uint64_t j10 = kind == 2 ? (uint64_t)v.j : 1023ull, b10 = kind == 2 ? (uint64_t)b : 1023ull;
                        const size_t o = (size_t)t * (size_t)cap + (size_t)p;
                        code_out[o] = kind | ((uint64_t)v.i << 2) | (j10 << 12) | ((uint64_t)a << 22) | (b10 << 32);
                        ratio_out[o] = (double)ratio;
                        contrib_out[o] = (double)contrib;
                    }
                }
                cnt += __popc(bal);
            }
        }
    }
    if (lane == 0) {
        count_out[t] = cnt;
        if (walked_out) {
            walked_out[2 * (size_t)t] = walked_s;
            walked_out[2 * (size_t)t + 1] = walked_d;
        }
        if (flag) atomicOr(status, flag);
    }
}

// Move update: one CTA per walker (Sec. III.B): diagonal energy, Jastrow sums, Fock sums, then the
// rank-1 (singles, opposite-spin doubles) or rank-2 Woodbury (same-spin doubles) update of G and
// AinvT, and the occupation lists, bits and orbital map.
template <typename real, bool kC>
__device__ __forceinline__ void apply_walker(const ListsView &L, const WalkerArgs &A, const double *__restrict__ J,
                                             const int w, const uint64_t *__restrict__ move_code,
                                             unsigned char *smraw, const CpsView &C = CpsView{}) {
    const Geo geo = make_geo(A.M, A.na, A.nb);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nt = blockDim.x, nwarp = nt >> 5;
    const uint64_t code = move_code[w];
    if (code == 0) return;
    const int M = geo.M, ne = geo.ne, N2 = 2 * M;
    uint16_t *pos = (uint16_t *)smraw;
    real *vec = (real *)(((uintptr_t)(pos + 2 * M) + 15) & ~(uintptr_t)15);
    // vec holds: ua[nmax], ub[nmax], gci[M], gcj[M], arow_i[nmax], arow_j[nmax]
    __shared__ double red[32];
    real *Gw = (real *)A.G + (size_t)w * geo.g_stride;
    real *Aw = (real *)A.AinvT + (size_t)w * geo.a_stride;
    real *Sw = (real *)A.S + (size_t)w * N2;
    uint16_t *occ = A.occ_list + (size_t)w * ne;
    uint16_t *virt = A.virt_list + (size_t)w * (2 * M - ne);
    uint32_t *bits = A.occ_bits_w + (size_t)w * 2 * geo.nw;
    uint16_t *posw = A.pos + (size_t)w * N2;
    for (int p = tid; p < N2; p += nt) pos[p] = posw[p];
    __syncthreads();
    const int kind = (int)(code & 3), I = (int)((code >> 2) & 1023), Jo = (int)((code >> 12) & 1023);
    const int Ao = (int)((code >> 22) & 1023), Bo = (int)((code >> 32) & 1023);
    // ---- correlator indices: every (changed orbital, covering correlator) adds its digit change
    if (kC && tid == 0) {
        uint16_t *ci = A.cps + (size_t)w * C.n_corr;
        const int chg[4] = {I, Ao, Jo, Bo};
        for (int x = 0; x < (kind == 2 ? 4 : 2); ++x) {
            const int sp = chg[x] >= M ? 1 : 0, site = chg[x] - sp * M, dg = ((x & 1) ? 1 : -1) * (1 + sp);
            for (int h = C.site_off[site]; h < C.site_off[site + 1]; ++h) {
                const uint32_t ent = C.site_ent[h];
                ci[ent >> 16] = (uint16_t)((int)ci[ent >> 16] + dg * (int)(ent & 0xFFFFu));
            }
        }
    }

    // ---- diagonal energy change (old occupation), FP64
    {
        auto D = [&](int p, int q) -> double {
            const int kp = p % M, kq = q % M;
            double d = L.Jd[(size_t)kp * M + kq];
            if ((p >= M) == (q >= M)) d -= L.Kd[(size_t)kp * M + kq];
            return d;
        };
        double part = 0.0;
        for (int t = tid; t < ne; t += nt) {
            const int K = (t < geo.na ? 0 : M) + occ[t];
            if (K != I) part += D(Ao, K) - D(I, K);
            if (kind == 2 && K != I && K != Jo) part += D(Bo, K) - D(Jo, K);
        }
        part = warp_sum_f64(part);
        if (lane == 0) red[warp] = part;
        __syncthreads();
        if (tid == 0) {
            double dE = L.hd[Ao % M] - L.hd[I % M];
            if (kind == 2) dE += L.hd[Bo % M] - L.hd[Jo % M] + D(Bo, Ao) - D(Jo, Ao);
            for (int k = 0; k < nwarp; ++k) dE += red[k];
            A.e_diag[w] += dE;
        }
    }
    // ---- Jastrow sums: S_p += J_pa [p != a] - J_pi [p != i]  (twice for doubles)
    for (int p = tid; p < N2; p += nt) {
        double d = 0.0;
        if (p != Ao) d += jget(J, N2, p, Ao);
        if (p != I) d -= jget(J, N2, p, I);
        if (kind == 2) {
            if (p != Bo) d += jget(J, N2, p, Bo);
            if (p != Jo) d -= jget(J, N2, p, Jo);
        }
        Sw[p] = (real)((double)Sw[p] + d);
    }
    // ---- Fock sums: each changed spin orbital k of spin t adds +-Tjk[k] to spin t, +-Tj[k] to the other
    {
        typedef typename Vec16<real>::type vec_t;
        constexpr int VE = Vec16<real>::n;
        const int64_t np = L.ns_pad, nvec = np / VE;
        vec_t *F0 = (vec_t *)((real *)A.F + (size_t)w * 2 * np), *F1 = F0 + nvec;
        const real *Tk = fock_table<real>(L, 1), *Tx = fock_table<real>(L, 0);
        const int nch = kind == 2 ? 4 : 2;
        const int chg[4] = {I, Ao, Jo, Bo};
        for (int64_t v = tid; v < nvec; v += nt) {
            vec_t f0 = F0[v], f1 = F1[v];
            for (int c = 0; c < nch; ++c) {
                const int p = chg[c];
                const real sgn = (c & 1) ? real(1) : real(-1);
                const int t = p >= M, k = p - t * M;
                const vec_t jk = __ldg((const vec_t *)(Tk + (size_t)k * np) + v);
                const vec_t jj = __ldg((const vec_t *)(Tx + (size_t)k * np) + v);
                if (t == 0) { vadd(f0, sgn, jk); vadd(f1, sgn, jj); }
                else { vadd(f1, sgn, jk); vadd(f0, sgn, jj); }
            }
            F0[v] = f0; F1[v] = f1;
        }
    }
    // ---- determinant tables: rank-1 per spin (singles, opposite-spin doubles) or rank-2
    //      Woodbury (same-spin doubles) on G and AinvT (Sherman-Morrison, Sec. III.B)
    const int nmax = geo.na > geo.nb ? geo.na : geo.nb, np4 = (nmax + 3) & ~3, mp4 = (M + 3) & ~3;
    real *ua = vec, *ub = ua + np4, *gci = ub + np4, *gcj = gci + mp4, *ari = gcj + mp4, *arj = ari + np4;
    int nsteps = 1;
    int sp[2], fr[2][2], to[2][2], rk[2];
    const int si = I >= M;
    if (kind == 1) { sp[0] = si; fr[0][0] = I - si * M; to[0][0] = Ao - si * M; rk[0] = 1; }
    else if (Jo / M == si) {   // same-spin double
        sp[0] = si; rk[0] = 2;
        fr[0][0] = I - si * M; to[0][0] = Ao - si * M; fr[0][1] = Jo - si * M; to[0][1] = Bo - si * M;
    } else {                   // opposite spin: alpha i->a, beta j->b
        nsteps = 2;
        sp[0] = 0; rk[0] = 1; fr[0][0] = I; to[0][0] = Ao;
        sp[1] = 1; rk[1] = 1; fr[1][0] = Jo - M; to[1][0] = Bo - M;
    }
    // The vectors of step st: ua/ub = R^-1 (G[(a,b),:] - E) with R = G[(a,b), (ci,cj)], the old
    // columns ci (cj) of G and rows ci (cj) of C_occ^-1.  u2, g2, a2 may be null for a rank-1 step
    // (then the second term of the update is zero).
    auto prep = [&](int st, real *u1, real *u2, real *g1, real *g2, real *a1, real *a2) {
        const int s = sp[st], n = geo.n(s), nv = M - n;
        const real *Gs = Gw + geo.g_off(s);
        const real *As = Aw + geo.a_off(s);
        const int ci = pos[s * M + fr[st][0]], sa = pos[s * M + to[st][0]] & 0x7FFF;
        int cj = 0, sb = 0;
        if (rk[st] == 2) { cj = pos[s * M + fr[st][1]]; sb = pos[s * M + to[st][1]] & 0x7FFF; }
        real r00 = Gs[(size_t)sa * n + ci], r01 = 0, r10 = 0, r11 = 1;
        if (rk[st] == 2) { r01 = Gs[(size_t)sa * n + cj]; r10 = Gs[(size_t)sb * n + ci]; r11 = Gs[(size_t)sb * n + cj]; }
        const real det = r00 * r11 - r01 * r10;
        const real i00 = r11 / det, i01 = -r01 / det, i10 = -r10 / det, i11 = r00 / det;
        for (int c = tid; c < n; c += nt) {
            const real va = Gs[(size_t)sa * n + c] - (c == ci ? (real)1 : (real)0);
            const real vb = rk[st] == 2 ? Gs[(size_t)sb * n + c] - (c == cj ? (real)1 : (real)0) : (real)0;
            u1[c] = i00 * va + i01 * vb;
            a1[c] = As[(size_t)ci * n + c];
            if (u2) {
                u2[c] = i10 * va + i11 * vb;
                a2[c] = rk[st] == 2 ? As[(size_t)cj * n + c] : (real)0;
            }
        }
        for (int r = tid; r < nv; r += nt) {
            real x = Gs[(size_t)r * n + ci], y = rk[st] == 2 ? Gs[(size_t)r * n + cj] : (real)0;
            if (r == sa) { x = 1; y = 0; }
            if (rk[st] == 2 && r == sb) { x = 0; y = 1; }
            g1[r] = x;
            if (g2) g2[r] = y;
        }
    };
    // G <- G - g1 u1^T - g2 u2^T (replaced rows taken as unit vectors), C_occ^-1 likewise
    auto update = [&](int st, const real *u1, const real *u2, const real *g1, const real *g2, const real *a1,
                      const real *a2) {
        const int s = sp[st], n = geo.n(s), nv = M - n;
        real *Gs = Gw + geo.g_off(s);
        real *As = Aw + geo.a_off(s);
        const int ci = pos[s * M + fr[st][0]], sa = pos[s * M + to[st][0]] & 0x7FFF;
        int cj = 0, sb = 0;
        if (rk[st] == 2) { cj = pos[s * M + fr[st][1]]; sb = pos[s * M + to[st][1]] & 0x7FFF; }
        typedef typename Vec16<real>::type vec_t;
        constexpr int VE = Vec16<real>::n;
        const bool rk2 = rk[st] == 2;
        if (n % VE == 0 && n > 0 && ((((uintptr_t)Gs) | ((uintptr_t)As)) & 15) == 0) {
            // 16-byte vectors: thread -> fixed column chunk cv, rows r0, r0 + rs, ...
            const int nvc = n / VE, cv = tid % nvc, r0 = tid / nvc, rs = nt / nvc, c0 = cv * VE;
            if (r0 < rs) {
                vec_t zero;
                real *ze = (real *)&zero;
#pragma unroll
                for (int q = 0; q < VE; ++q) ze[q] = real(0);
                const vec_t u = *(const vec_t *)(u1 + c0), v = u2 ? *(const vec_t *)(u2 + c0) : zero;
                vec_t *Gv = (vec_t *)Gs;
#pragma unroll 4
                for (int r = r0; r < nv; r += rs) {
                    vec_t o = Gv[(size_t)r * nvc + cv];
                    if (r == sa || (rk2 && r == sb)) {   // replaced row: old value is a unit vector
                        const int cu = r == sa ? ci : cj;
                        real *oe = (real *)&o;
#pragma unroll
                        for (int q = 0; q < VE; ++q) oe[q] = (c0 + q == cu) ? real(1) : real(0);
                    }
                    Gv[(size_t)r * nvc + cv] = vfma2(o, g1[r], u, g2 ? g2[r] : real(0), v);
                }
                const vec_t b1 = *(const vec_t *)(a1 + c0), b2 = a2 ? *(const vec_t *)(a2 + c0) : zero;
                vec_t *Av = (vec_t *)As;
#pragma unroll 4
                for (int c = r0; c < n; c += rs)
                    Av[(size_t)c * nvc + cv] = vfma2(Av[(size_t)c * nvc + cv], u1[c], b1, u2 ? u2[c] : real(0), b2);
            }
        } else {
            for (size_t t = tid; t < (size_t)nv * n; t += nt) {
                const int r = (int)(t / n), c = (int)(t % n);
                real old = Gs[t];
                if (r == sa) old = (c == ci) ? (real)1 : (real)0;
                if (rk2 && r == sb) old = (c == cj) ? (real)1 : (real)0;
                Gs[t] = old - g1[r] * u1[c] - (g2 ? g2[r] : real(0)) * (u2 ? u2[c] : real(0));
            }
            for (size_t t = tid; t < (size_t)n * n; t += nt) {
                const int c = (int)(t / n), x = (int)(t % n);
                As[t] = As[t] - u1[c] * a1[x] - (u2 ? u2[c] : real(0)) * (a2 ? a2[x] : real(0));
            }
        }
    };
    // occupation list, virtual list, orbital map and bit string of step st (one thread)
    auto relist = [&](int st) {
        const int s = sp[st];
        uint16_t *occs = occ + (s ? geo.na : 0);
        uint16_t *virts = virt + (s ? geo.nv_a : 0);
        const int ci = pos[s * M + fr[st][0]], sa = pos[s * M + to[st][0]] & 0x7FFF;
        int cj = 0, sb = 0;
        if (rk[st] == 2) { cj = pos[s * M + fr[st][1]]; sb = pos[s * M + to[st][1]] & 0x7FFF; }
        occs[ci] = (uint16_t)to[st][0];
        virts[sa] = (uint16_t)fr[st][0];
        posw[s * M + to[st][0]] = (uint16_t)ci;
        posw[s * M + fr[st][0]] = (uint16_t)(0x8000 | sa);
        if (rk[st] == 2) {
            occs[cj] = (uint16_t)to[st][1];
            virts[sb] = (uint16_t)fr[st][1];
            posw[s * M + to[st][1]] = (uint16_t)cj;
            posw[s * M + fr[st][1]] = (uint16_t)(0x8000 | sb);
        }
        uint32_t *bw = bits + s * geo.nw;
        for (int k = 0; k < rk[st]; ++k) {
            const int f = fr[st][k], tt = to[st][k];
            bw[f >> 5] &= ~(1u << (f & 31));
            bw[tt >> 5] |= 1u << (tt & 31);
        }
    };
    __syncthreads();
    if (nsteps == 2) {   // opposite-spin double: the two spins' rank-1 updates share the phases
        prep(0, ua, nullptr, gci, nullptr, ari, nullptr);
        prep(1, ub, nullptr, gcj, nullptr, arj, nullptr);
        __syncthreads();
        update(0, ua, nullptr, gci, nullptr, ari, nullptr);
        update(1, ub, nullptr, gcj, nullptr, arj, nullptr);
        __syncthreads();
        if (tid == 0) { relist(0); relist(1); }
    } else {
        prep(0, ua, ub, gci, gcj, ari, arj);
        __syncthreads();
        update(0, ua, ub, gci, gcj, ari, arj);
        __syncthreads();
        if (tid == 0) relist(0);
    }
}


// 256 threads per walker; six resident CTAs per SM (<= 40 registers): the update is bound by HBM
// latency between its barrier-separated phases, so more walkers in flight per SM pay (12 % faster
// than four per SM at H160, with a few spilled registers)
template <typename real, bool kC>
__global__ void __launch_bounds__(256, 6)
k_ctmc_apply(ListsView L, WalkerArgs A, CpsView C, const double *__restrict__ J, const uint64_t *__restrict__ move_code) {
    extern __shared__ __align__(16) unsigned char smraw[];
    apply_walker<real, kC>(L, A, J, blockIdx.x, move_code, smraw, C);
}

template <typename real>
__global__ void __launch_bounds__(512)
k_ctmc_apply_batched(const SysDesc *__restrict__ sys, int n_sys) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int t = blockIdx.x;
    int k = 0;
    while (k + 1 < n_sys && sys[k + 1].w_begin <= t) ++k;
    const SysDesc &d = sys[k];
    apply_walker<real, false>(d.L, d.A, d.J, t - d.w_begin, d.move_code, smraw);
}

}  // namespace

// per-warp entry queues of the local-energy kernel: 2 x 64 codes of 4 bytes
static size_t eloc_queue_bytes(int threads) { return (size_t)(threads / 32) * 128 * sizeof(uint32_t); }

static WalkerArgs make_args(vmc_walkers *Wk) {
    WalkerArgs A;
    A.W = Wk->W; A.M = Wk->M; A.na = Wk->n_alpha; A.nb = Wk->n_beta;
    A.occ_bits = Wk->occ_bits; A.occ_bits_w = Wk->occ_bits;
    A.occ_list = Wk->occ_list; A.virt_list = Wk->virt_list; A.pos = Wk->pos;
    A.G = Wk->G; A.AinvT = Wk->AinvT; A.S = Wk->S; A.F = Wk->F; A.e_diag = Wk->e_diag;
    A.rng = Wk->rng_counter;
    A.cps = Wk->cps_state;
    return A;
}

template <typename real, int kT>
static cudaError_t eloc_launch_t(const vmc_ctx *ctx, int W, size_t smem, const ListsView &L, const WalkerArgs &A,
                                 const CpsView &C, double *e_loc, double *t_res, u128 *rates) {
    cudaError_t e;
    if (C.n_corr) {
        e = cudaFuncSetAttribute(k_local_energy_cps<real, kT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            k_local_energy_cps<real, kT><<<W, kT, smem, ctx->stream>>>(L, A, C, e_loc, t_res, rates, ctx->d_status);
        return e;
    }
    e = cudaFuncSetAttribute(k_local_energy<real, kT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) k_local_energy<real, kT><<<W, kT, smem, ctx->stream>>>(L, A, e_loc, t_res, rates, ctx->d_status);
    return e;
}
template <typename real>
static cudaError_t eloc_launch(const vmc_ctx *ctx, int W, size_t smem, const ListsView &L, const WalkerArgs &A,
                               const CpsView &C, double *e_loc, double *t_res, u128 *rates) {
    switch (ctx->eloc_threads) {
    case 128: return eloc_launch_t<real, 128>(ctx, W, smem, L, A, C, e_loc, t_res, rates);
    case 256: return eloc_launch_t<real, 256>(ctx, W, smem, L, A, C, e_loc, t_res, rates);
    case 384: return eloc_launch_t<real, 384>(ctx, W, smem, L, A, C, e_loc, t_res, rates);
    default: return eloc_launch_t<real, 512>(ctx, W, smem, L, A, C, e_loc, t_res, rates);
    }
}
template <typename real, int kT>
static cudaError_t eloc_batched_launch_t(const vmc_ctx *ctx, int nsm, size_t se, const SysDesc *tab, int n, int total) {
    int per_sm = 0;
    cudaError_t e = cudaFuncSetAttribute(k_local_energy_batched<real, kT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)se);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_local_energy_batched<real, kT>, kT, se);
    if (e == cudaSuccess)
        k_local_energy_batched<real, kT><<<std::max(1, per_sm) * nsm, kT, se, ctx->stream>>>(tab, n, total, ctx->d_queue,
                                                                                            ctx->d_status);
    return e;
}
template <typename real>
static cudaError_t eloc_batched_launch(const vmc_ctx *ctx, int nsm, size_t se, const SysDesc *tab, int n, int total) {
    switch (ctx->eloc_threads) {
    case 128: return eloc_batched_launch_t<real, 128>(ctx, nsm, se, tab, n, total);
    case 256: return eloc_batched_launch_t<real, 256>(ctx, nsm, se, tab, n, total);
    case 384: return eloc_batched_launch_t<real, 384>(ctx, nsm, se, tab, n, total);
    default: return eloc_batched_launch_t<real, 512>(ctx, nsm, se, tab, n, total);
    }
}

vmc_status launch_local_energy(vmc_ctx *ctx, const vmc_lists *L, vmc_walkers *Wk, const CpsView &C, double *e_loc,
                               double *t_res, u128 *rates, int n_groups) {
    const int M = Wk->M;
    (void)n_groups;
    const size_t esz = Wk->precision == VMC_FP64 ? 8 : 4;
    const int na = Wk->n_alpha, nb = Wk->n_beta;
    const size_t gpad = (size_t)(M - na) * (na + 1) + (size_t)(M - nb) * (nb + 1);
    // correlator product: 1/c per correlator (padded to 4) and a 16-bit index per correlator
    const size_t cps = C.n_corr ? esz * (size_t)((C.n_corr + 3) & ~3) + 4 * (2 * (size_t)C.n_corr + 1) +
                                      4 * ((size_t)M + 1) + 4 * (size_t)C.nnz
                                : 0;
    const size_t smem = esz * (gpad + 2 * (size_t)M) + 2 * (2 * (size_t)M) + 16 + eloc_queue_bytes(ctx->eloc_threads) + cps;
    if (smem > 200 * 1024) return set_err(ctx, VMC_ERR_ARG, "walker G table does not fit in shared memory");
    WalkerArgs A = make_args(Wk);
    cudaError_t e = Wk->precision == VMC_FP64
                              ? eloc_launch<double>(ctx, Wk->W, smem, L->view, A, C, e_loc, t_res, rates)
                              : eloc_launch<float>(ctx, Wk->W, smem, L->view, A, C, e_loc, t_res, rates);
    ctx->launches += 1;
    if (e == cudaSuccess) e = cudaGetLastError();
    return cuda_check(ctx, e, "k_local_energy");
}

template <typename real, bool kC>
static cudaError_t ctmc_launch(vmc_ctx *ctx, const vmc_lists *L, const vmc_params *P, const WalkerArgs &A,
                               const CpsView &C, int W, size_t smem, uint64_t seed, const u128 *rates,
                               uint64_t *move_code) {
    const int sel_blocks = (W + VMC_WARPS - 1) / VMC_WARPS;
    k_ctmc_select<real, kC><<<sel_blocks, VMC_THREADS, 0, ctx->stream>>>(L->view, A, C, rates, seed, move_code,
                                                                         ctx->d_status);
    cudaError_t e = cudaFuncSetAttribute(k_ctmc_apply<real, kC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) k_ctmc_apply<real, kC><<<W, VMC_THREADS, smem, ctx->stream>>>(L->view, A, C, P->J, move_code);
    return e;
}

vmc_status launch_ctmc_step(vmc_ctx *ctx, const vmc_lists *L, const vmc_params *P, vmc_walkers *Wk,
                            uint64_t seed, const u128 *rates, int n_groups, uint64_t *move_code) {
    const int M = Wk->M;
    (void)n_groups;
    const int nmax = Wk->n_alpha > Wk->n_beta ? Wk->n_alpha : Wk->n_beta;
    const size_t esz = Wk->precision == VMC_FP64 ? 8 : 4;
    const size_t smem = 2 * (2 * (size_t)M) + 32 + esz * (4 * (size_t)((nmax + 3) & ~3) + 2 * (size_t)((M + 3) & ~3));
    WalkerArgs A = make_args(Wk);
    const CpsView C = cps_view(P);
    cudaError_t e;
    if (Wk->precision == VMC_FP64)
        e = C.n_corr ? ctmc_launch<double, true>(ctx, L, P, A, C, Wk->W, smem, seed, rates, move_code)
                     : ctmc_launch<double, false>(ctx, L, P, A, C, Wk->W, smem, seed, rates, move_code);
    else
        e = C.n_corr ? ctmc_launch<float, true>(ctx, L, P, A, C, Wk->W, smem, seed, rates, move_code)
                     : ctmc_launch<float, false>(ctx, L, P, A, C, Wk->W, smem, seed, rates, move_code);
    ctx->launches += 2;
    if (e == cudaSuccess) e = cudaGetLastError();
    return cuda_check(ctx, e, "k_ctmc_select/k_ctmc_apply");
}

// ---------------------------------------------------------------------------------- batches
static size_t eloc_smem_bytes(const vmc_lists *L, const vmc_walkers *Wk, int threads) {
    const size_t esz = Wk->precision == VMC_FP64 ? 8 : 4;
    const int M = Wk->M, na = Wk->n_alpha, nb = Wk->n_beta;
    const size_t gpad = (size_t)(M - na) * (na + 1) + (size_t)(M - nb) * (nb + 1);
    (void)L;
    return esz * (gpad + 2 * (size_t)M) + 2 * (2 * (size_t)M) + 16 + eloc_queue_bytes(threads);
}

static size_t apply_smem_bytes(const vmc_walkers *Wk) {
    const int M = Wk->M, nmax = Wk->n_alpha > Wk->n_beta ? Wk->n_alpha : Wk->n_beta;
    const size_t esz = Wk->precision == VMC_FP64 ? 8 : 4;
    return 2 * (2 * (size_t)M) + 32 + esz * (4 * (size_t)((nmax + 3) & ~3) + 2 * (size_t)((M + 3) & ~3));
}

// Builds (and uploads when changed) the descriptor table of a batch, most expensive systems
// first.  Also sizes the shared rate store.  Outputs: total walkers, max shared memory.
static vmc_status prepare_batch(vmc_ctx *ctx, int n, const vmc_batch_item *items, int *total,
                                size_t *smem_eloc, size_t *smem_apply, int *precision) {
    extern vmc_status lists_set_eps(vmc_ctx *, vmc_lists *, double);
    if (n < 1 || n > 64 || !items) return set_err(ctx, VMC_ERR_ARG, "1 to 64 batch items");
    std::vector<int> order(n);
    std::vector<double> cost(n);
    for (int k = 0; k < n; ++k) {
        const vmc_batch_item &it = items[k];
        if (!it.lists || !it.params || !it.walkers || !it.d_e_loc || !it.d_t_res || !it.d_move_code)
            return set_err(ctx, VMC_ERR_ARG, "null batch item field");
        if (it.walkers->precision != items[0].walkers->precision)
            return set_err(ctx, VMC_ERR_ARG, "batch items must share the precision");
        if (it.walkers->M != it.lists->M) return set_err(ctx, VMC_ERR_ARG, "lists and walkers disagree on M");
        if (!(it.eps_run >= it.lists->eps_build)) return set_err(ctx, VMC_ERR_ARG, "eps_run below the build eps");
        vmc_status st = lists_set_eps(ctx, const_cast<vmc_lists *>(it.lists), it.eps_run);
        if (st) return st;
        order[k] = k;
        const vmc_lists *L = it.lists;
        cost[k] = (double)(L->ns + 2 * L->nds + L->ndo) * (it.walkers->n_alpha + it.walkers->n_beta) / (2.0 * L->M) +
                  (double)walker_stride_G(it.walkers->M, it.walkers->n_alpha, it.walkers->n_beta);
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    size_t rates_total = 0;
    std::vector<size_t> rate_off(n);
    int tot = 0;
    size_t se = 0, sa = 0;
    for (int k = 0; k < n; ++k) {
        const vmc_batch_item &it = items[order[k]];
        rate_off[k] = rates_total;
        rates_total += rate_store_units(it.walkers->W, it.lists->view.n_groups);
        tot += it.walkers->W;
        se = std::max(se, eloc_smem_bytes(it.lists, it.walkers, ctx->eloc_threads));
        sa = std::max(sa, apply_smem_bytes(it.walkers));
    }
    if (rates_total * sizeof(u128) > ctx->rates_bytes) {
        if (ctx->rates) { cudaStreamSynchronize(ctx->stream); cudaFree(ctx->rates); ctx->rates = nullptr; }
        cudaError_t e = cudaMalloc(&ctx->rates, rates_total * sizeof(u128));
        if (e != cudaSuccess) { ctx->rates_bytes = 0; return cuda_check(ctx, e, "batched rate store"); }
        ctx->rates_bytes = rates_total * sizeof(u128);
    }
    std::string tab(sizeof(SysDesc) * n, '\0');
    SysDesc *d = (SysDesc *)&tab[0];
    int wb = 0;
    for (int k = 0; k < n; ++k) {
        const vmc_batch_item &it = items[order[k]];
        d[k].L = it.lists->view;
        d[k].A = make_args(it.walkers);
        d[k].J = it.params->J;
        d[k].e_loc = it.d_e_loc;
        d[k].t_res = it.d_t_res;
        d[k].rates = (u128 *)ctx->rates + rate_off[k];
        d[k].move_code = it.d_move_code;
        d[k].w_begin = wb;
        wb += it.walkers->W;
    }
    if (tab != ctx->batch_host) {
        if (tab.size() > ctx->batch_desc_bytes) {
            if (ctx->batch_desc) { cudaStreamSynchronize(ctx->stream); cudaFree(ctx->batch_desc); }
            cudaError_t e = cudaMalloc(&ctx->batch_desc, tab.size());
            if (e != cudaSuccess) { ctx->batch_desc = nullptr; ctx->batch_desc_bytes = 0; return cuda_check(ctx, e, "batch table"); }
            ctx->batch_desc_bytes = tab.size();
        }
        if (!ctx->d_queue) {
            cudaError_t e = cudaMalloc(&ctx->d_queue, sizeof(int));
            if (e != cudaSuccess) { ctx->d_queue = nullptr; return cuda_check(ctx, e, "batch queue"); }
        }
        cudaError_t e = cudaMemcpyAsync(ctx->batch_desc, tab.data(), tab.size(), cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return cuda_check(ctx, e, "batch table upload");
        ctx->batch_host = tab;
    }
    *total = tot;
    *smem_eloc = se;
    *smem_apply = sa;
    *precision = items[0].walkers->precision;
    return VMC_OK;
}

static std::string batch_signature(int n, const vmc_batch_item *items) {
    std::string sig;
    for (int k = 0; k < n; ++k) sig.append((const char *)&items[k].walkers->G, sizeof(void *));
    return sig;
}

vmc_status launch_local_energy_batch(vmc_ctx *ctx, int n, const vmc_batch_item *items) {
    int total = 0, prec = 0;
    size_t se = 0, sa = 0;
    vmc_status st = prepare_batch(ctx, n, items, &total, &se, &sa, &prec);
    if (st) return st;
    if (se > 200 * 1024) return set_err(ctx, VMC_ERR_ARG, "walker G table does not fit in shared memory");
    cudaError_t e = cudaMemsetAsync(ctx->d_queue, 0, sizeof(int), ctx->stream);
    int dev = 0, nsm = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const SysDesc *tab = (const SysDesc *)ctx->batch_desc;
    if (e == cudaSuccess)
        e = prec == VMC_FP64 ? eloc_batched_launch<double>(ctx, nsm, se, tab, n, total)
                             : eloc_batched_launch<float>(ctx, nsm, se, tab, n, total);
    ctx->launches += 1;
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(ctx, e, "k_local_energy_batched");
    ctx->rates_batch = batch_signature(n, items);
    ctx->rates_valid = 0;
    return VMC_OK;
}

vmc_status launch_ctmc_step_batch(vmc_ctx *ctx, int n, const vmc_batch_item *items, uint64_t seed) {
    if (ctx->rates_batch.empty() || ctx->rates_batch != batch_signature(n, items))
        return set_err(ctx, VMC_ERR_ARG, "vmc_local_energy_batch must precede vmc_ctmc_step_batch on the same items");
    int total = 0, prec = 0;
    size_t se = 0, sa = 0;
    vmc_status st = prepare_batch(ctx, n, items, &total, &se, &sa, &prec);
    if (st) return st;
    const SysDesc *tab = (const SysDesc *)ctx->batch_desc;
    const int sel_blocks = (total + 7) / 8;
    cudaError_t e;
    if (prec == VMC_FP64) {
        k_ctmc_select_batched<double><<<sel_blocks, 256, 0, ctx->stream>>>(tab, n, total, seed, ctx->d_status);
        e = cudaFuncSetAttribute(k_ctmc_apply_batched<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sa);
        if (e == cudaSuccess) k_ctmc_apply_batched<double><<<total, 256, sa, ctx->stream>>>(tab, n);
    } else {
        k_ctmc_select_batched<float><<<sel_blocks, 256, 0, ctx->stream>>>(tab, n, total, seed, ctx->d_status);
        e = cudaFuncSetAttribute(k_ctmc_apply_batched<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sa);
        if (e == cudaSuccess) k_ctmc_apply_batched<float><<<total, 256, sa, ctx->stream>>>(tab, n);
    }
    ctx->launches += 2;
    if (e == cudaSuccess) e = cudaGetLastError();
    ctx->rates_batch.clear();
    return cuda_check(ctx, e, "k_ctmc_*_batched");
}

vmc_status launch_screened_moves(vmc_ctx *ctx, const vmc_lists *L, const vmc_walkers *Wk, const CpsView &C,
                                 int w_begin, int n_w, int64_t cap, uint64_t *code, double *ratio, double *contrib,
                                 int64_t *count, int64_t *walked) {
    WalkerArgs A = make_args(const_cast<vmc_walkers *>(Wk));
    const int blocks = (n_w + VMC_WARPS - 1) / VMC_WARPS;
#define VMC_MOVES(real, kc)                                                                                      \
    k_screened_moves<real, kc><<<blocks, VMC_THREADS, 0, ctx->stream>>>(L->view, A, C, w_begin, n_w, cap, code, \
                                                                       ratio, contrib, count, walked, ctx->d_status)
    if (Wk->precision == VMC_FP64) {
        if (C.n_corr) VMC_MOVES(double, true); else VMC_MOVES(double, false);
    } else {
        if (C.n_corr) VMC_MOVES(float, true); else VMC_MOVES(float, false);
    }
#undef VMC_MOVES
    ctx->launches += 1;
    return cuda_check(ctx, cudaGetLastError(), "k_screened_moves");
}
