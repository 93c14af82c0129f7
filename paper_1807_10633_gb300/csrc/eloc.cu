// Screened local energy (Sec. II.A, Eq. eloc:hci) and the rejection-free CTMC move (Sec. II.B).
//
// One CTA per walker.  The walker's G (virtual rows only), exp(S) and the orbital -> column /
// slot map are staged in shared memory; the screened lists (shared by all walkers, L2-resident)
// are streamed per occupied pair.  Work units in canonical order are: the walker's occupied spin
// orbitals (singles), then its occupied pairs (i<j) lexicographically (doubles).  Units are taken
// 32 at a time ("groups"); inside a group the lists of the 32 units are concatenated and walked
// one entry per lane, so short lists do not idle lanes.  Each group's CTMC rates are summed as
// exact 128-bit fixed-point integers (order independent) and stored; the CTMC kernel re-walks
// only the chosen group.  Every product that enters a rate uses explicitly rounded intrinsics so
// the two kernels compute bit-identical rates.
#include <math.h>

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

template <typename real> __device__ __forceinline__ real lw_single(const ListsView &L, int s, uint32_t e);
template <> __device__ __forceinline__ double lw_single<double>(const ListsView &L, int s, uint32_t e) { return L.s_wd[(size_t)s * L.ns + e]; }
template <> __device__ __forceinline__ float lw_single<float>(const ListsView &L, int s, uint32_t e) { return L.s_wf[(size_t)s * L.ns + e]; }
template <typename real> __device__ __forceinline__ real lw_same(const ListsView &L, int s, uint32_t e);
template <> __device__ __forceinline__ double lw_same<double>(const ListsView &L, int s, uint32_t e) { return L.ds_wd[(size_t)s * L.nds + e]; }
template <> __device__ __forceinline__ float lw_same<float>(const ListsView &L, int s, uint32_t e) { return L.ds_wf[(size_t)s * L.nds + e]; }
template <typename real> __device__ __forceinline__ real lv_same(const ListsView &L, uint32_t e);
template <> __device__ __forceinline__ double lv_same<double>(const ListsView &L, uint32_t e) { return L.ds_vd[e]; }
template <> __device__ __forceinline__ float lv_same<float>(const ListsView &L, uint32_t e) { return L.ds_vf[e]; }
template <typename real> __device__ __forceinline__ real lw_opp(const ListsView &L, uint32_t e);
template <> __device__ __forceinline__ double lw_opp<double>(const ListsView &L, uint32_t e) { return L.do_wd[e]; }
template <> __device__ __forceinline__ float lw_opp<float>(const ListsView &L, uint32_t e) { return L.do_wf[e]; }
template <typename real> __device__ __forceinline__ real lv_opp(const ListsView &L, uint32_t e);
template <> __device__ __forceinline__ double lv_opp<double>(const ListsView &L, uint32_t e) { return L.do_vd[e]; }
template <> __device__ __forceinline__ float lv_opp<float>(const ListsView &L, uint32_t e) { return L.do_vf[e]; }

// Walker arrays (global) and geometry.
struct WalkerArgs {
    int W, M, na, nb;
    const uint32_t *occ_bits;
    uint16_t *occ_list, *virt_list;
    uint32_t *occ_bits_w;
    void *G, *AinvT, *S;
    double *F, *e_diag;
    uint64_t *rng;
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
    real einv;     // 1 / (E_i E_j)   (1 / E_i for singles)
};

// Shared-memory view of one walker used by the entry evaluation.
template <typename real>
struct View {
    const uint16_t *pos;   // [2M]: occupied -> column, virtual -> 0x8000 | slot
    const real *G;         // walker G, shared or global, layout as Geo
    const real *E;         // [2M] exp(S) (nullptr: compute from S on the fly)
    const real *S;         // walker S in global (used when E == nullptr)
    const double *F;       // walker F [2][ns]
    Geo geo;
    __device__ real Ev(int p) const { return E ? E[p] : rexp(S[p]); }
};

template <typename real>
__device__ __forceinline__ void setup_unit(const ListsView &L, const View<real> &V, int kind_grp,
                                           int x, int y, const uint16_t *socc, Unit<real> &u) {
    const int M = V.geo.M;
    if (kind_grp == 0) {
        const int i = socc[y];
        const int s = i >= M, pi = i - s * M;
        u.kind = 0; u.cls = s; u.i = i; u.j = -1;
        u.base = L.s_off[pi]; u.len = L.s_len[pi];
        u.ci = V.pos[i]; u.cj = 0;
        u.einv = rrcp(V.Ev(i));
    } else {
        const int i = socc[x], j = socc[y];
        const int si = i >= M, sj = j >= M, pi = i - si * M, pj = j - sj * M;
        u.i = i; u.j = j;
        u.ci = V.pos[i]; u.cj = V.pos[j];
        u.einv = rrcp(rmul(V.Ev(i), V.Ev(j)));
        if (si == sj) {
            const int t = tri_index(pi, pj, M);
            u.kind = 1; u.cls = si;
            u.base = L.ds_off[t]; u.len = L.ds_len[t];
        } else {
            const int t = pi * M + pj;
            u.kind = 2; u.cls = 0;
            u.base = L.do_off[t]; u.len = L.do_len[t];
        }
    }
}

// Evaluate list entry `idx` of unit u.  Returns false if the target orbital(s) are occupied.
// On true: ratio = psi(m)/psi(n) (in-place replacement convention, the fermionic phases of H
// and of the ratio cancel) and contrib = H_nm * ratio.
template <typename real>
__device__ __forceinline__ bool eval_entry(const ListsView &L, const View<real> &V, const Unit<real> &u,
                                           uint32_t idx, real &ratio, real &contrib, int &A, int &B) {
    const int M = V.geo.M;
    if (u.kind == 0) {
        const int s = u.cls;
        const int a = L.s_a[idx];
        const uint16_t pa = V.pos[s * M + a];
        if (!(pa & 0x8000)) return false;
        const int n = V.geo.n(s);
        const real g = V.G[V.geo.g_off(s) + (size_t)(pa & 0x7FFF) * n + u.ci];
        const real r = rmul(rmul(rmul(g, lw_single<real>(L, s, idx)), V.Ev(s * M + a)), u.einv);
        ratio = r;
        contrib = rmul((real)V.F[(size_t)s * L.ns + idx], r);
        A = s * M + a; B = -1;
        return true;
    }
    if (u.kind == 1) {
        const int s = u.cls;
        const uint32_t ab = L.ds_ab[idx];
        const int a = ab & 0xFFFF, b = ab >> 16;
        const uint16_t pa = V.pos[s * M + a], pb = V.pos[s * M + b];
        if (!(pa & pb & 0x8000)) return false;
        const int n = V.geo.n(s);
        const real *Gs = V.G + V.geo.g_off(s);
        const real *ra = Gs + (size_t)(pa & 0x7FFF) * n, *rb = Gs + (size_t)(pb & 0x7FFF) * n;
        const real minor = rsub(rmul(ra[u.ci], rb[u.cj]), rmul(ra[u.cj], rb[u.ci]));
        const real r = rmul(rmul(rmul(rmul(minor, lw_same<real>(L, s, idx)), V.Ev(s * M + a)),
                                 V.Ev(s * M + b)), u.einv);
        ratio = r;
        contrib = rmul(lv_same<real>(L, idx), r);
        A = s * M + a; B = s * M + b;
        return true;
    }
    const uint32_t ab = L.do_ab[idx];
    const int a = ab & 0xFFFF, b = ab >> 16;
    const uint16_t pa = V.pos[a], pb = V.pos[M + b];
    if (!(pa & pb & 0x8000)) return false;
    const real ga = V.G[(size_t)(pa & 0x7FFF) * V.geo.na + u.ci];
    const real gb = V.G[V.geo.g_off(1) + (size_t)(pb & 0x7FFF) * V.geo.nb + u.cj];
    const real r = rmul(rmul(rmul(rmul(rmul(ga, gb), lw_opp<real>(L, idx)), V.Ev(a)), V.Ev(M + b)), u.einv);
    ratio = r;
    contrib = rmul(lv_opp<real>(L, idx), r);
    A = a; B = M + b;
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

// Number of groups and the start of each row x of the doubles groups.
__host__ __device__ inline int chunks_of_row(int ne, int x) { return (ne - 1 - x + 31) / 32; }

// Decode group g -> (kind_grp, x, y0).  gstart[x] = first doubles group of row x.
__device__ __forceinline__ void decode_group(int g, int ne, const uint16_t *gstart, int &kg, int &x, int &y0) {
    const int gs = (ne + 31) / 32;
    if (g < gs) { kg = 0; x = -1; y0 = g * 32; return; }
    const int gd = g - gs;
    int lo = 0, hi = ne - 2;   // largest x with gstart[x] <= gd
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (gstart[mid] <= gd) lo = mid; else hi = mid - 1;
    }
    kg = 1; x = lo; y0 = x + 1 + 32 * (gd - gstart[x]);
}

// Prologue shared by both kernels: orbital -> column/slot map, sorted occupied spin orbitals,
// group row starts.
__device__ void build_maps(const Geo &geo, const uint16_t *occ, const uint16_t *virt, const uint32_t *bits,
                           uint16_t *pos, uint16_t *socc, uint16_t *gstart) {
    const int tid = threadIdx.x, nt = blockDim.x, M = geo.M;
    for (int c = tid; c < geo.ne; c += nt) {
        const int s = c < geo.na ? 0 : 1;
        const int col = c - (s ? geo.na : 0);
        pos[s * M + occ[c]] = (uint16_t)col;
    }
    const int nvt = 2 * M - geo.ne;
    for (int t = tid; t < nvt; t += nt) {
        const int s = t < geo.nv_a ? 0 : 1;
        const int slot = t - (s ? geo.nv_a : 0);
        pos[s * M + virt[t]] = (uint16_t)(0x8000 | slot);
    }
    // rank of each occupied spin orbital among all occupied spin orbitals (alpha block first)
    for (int p = tid; p < 2 * M; p += nt) {
        const int s = p >= M, k = p - s * M;
        const uint32_t *bw = bits + s * geo.nw;
        if (!((bw[k >> 5] >> (k & 31)) & 1u)) continue;
        int r = s ? geo.na : 0;
        for (int q = 0; q < (k >> 5); ++q) r += __popc(bw[q]);
        r += __popc(bw[k >> 5] & ((1u << (k & 31)) - 1u));
        socc[r] = (uint16_t)p;
    }
    if (tid == 0) {
        int acc = 0;
        for (int x = 0; x + 1 < geo.ne; ++x) { gstart[x] = (uint16_t)acc; acc += chunks_of_row(geo.ne, x); }
    }
}

template <typename real> struct AccT { typedef double type; };
template <> struct AccT<float> { typedef float type; };

template <typename real>
__global__ void __launch_bounds__(VMC_THREADS)
k_local_energy(ListsView L, WalkerArgs A, double *__restrict__ e_loc, double *__restrict__ t_res,
               u128 *__restrict__ rates, int n_groups, unsigned *status) {
    const Geo geo = make_geo(A.M, A.na, A.nb);
    const int w = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nt = blockDim.x;
    const int M = geo.M, ne = geo.ne;
    extern __shared__ __align__(16) unsigned char smraw[];
    real *sG = (real *)smraw;
    real *sE = sG + geo.g_stride;
    uint16_t *pos = (uint16_t *)(sE + 2 * M);
    uint16_t *socc = pos + 2 * M;
    uint16_t *gstart = socc + ne;
    // per-warp unit tables
    __shared__ uint32_t u_base[VMC_WARPS][32], u_off[VMC_WARPS][33];
    __shared__ uint8_t u_kind[VMC_WARPS][32], u_cls[VMC_WARPS][32];
    __shared__ uint16_t u_ci[VMC_WARPS][32], u_cj[VMC_WARPS][32];
    __shared__ real u_einv[VMC_WARPS][32];
    __shared__ double red_e[VMC_WARPS];
    __shared__ u128 red_q[VMC_WARPS];

    // ---- prologue: stage G (vectorised), exp(S), maps
    {
        const real *Gw = (const real *)A.G + (size_t)w * geo.g_stride;
        const size_t nbytes = geo.g_stride * sizeof(real);
        const int4 *src = (const int4 *)Gw;
        int4 *dst = (int4 *)sG;
        const size_t n16 = nbytes / 16;
        if ((((uintptr_t)Gw) & 15) == 0) {
            for (size_t t = tid; t < n16; t += nt) dst[t] = src[t];
            for (size_t t = n16 * 16 / sizeof(real) + tid; t < geo.g_stride; t += nt) sG[t] = Gw[t];
        } else {
            for (size_t t = tid; t < geo.g_stride; t += nt) sG[t] = Gw[t];
        }
        const real *Sw = (const real *)A.S + (size_t)w * 2 * M;
        for (int p = tid; p < 2 * M; p += nt) sE[p] = rexp(Sw[p]);
        build_maps(geo, A.occ_list + (size_t)w * ne, A.virt_list + (size_t)w * (2 * M - ne),
                   A.occ_bits + (size_t)w * 2 * geo.nw, pos, socc, gstart);
    }
    __syncthreads();

    View<real> V;
    V.pos = pos; V.G = sG; V.E = sE; V.S = nullptr; V.F = A.F + (size_t)w * 2 * L.ns; V.geo = geo;
    typedef typename AccT<real>::type acc_t;
    double e_acc = 0.0;
    u128 q_tot = 0;
    unsigned flag = 0;

    for (int g = warp; g < n_groups; g += VMC_WARPS) {
        int kg, x, y0;
        decode_group(g, ne, gstart, kg, x, y0);
        const int y = y0 + lane;
        Unit<real> u;
        u.len = 0;
        if (y < ne) {
            setup_unit<real>(L, V, kg, x, y, socc, u);
            u_base[warp][lane] = u.base;
            u_kind[warp][lane] = (uint8_t)u.kind;
            u_cls[warp][lane] = (uint8_t)u.cls;
            u_ci[warp][lane] = (uint16_t)u.ci;
            u_cj[warp][lane] = (uint16_t)u.cj;
            u_einv[warp][lane] = u.einv;
        }
        // exclusive scan of the list lengths
        uint32_t incl = u.len;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t o = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += o;
        }
        u_off[warp][lane] = incl - u.len;
        if (lane == 31) u_off[warp][32] = incl;
        __syncwarp();
        const uint32_t total = u_off[warp][32];
        acc_t e_grp = 0;
        u128 q_grp = 0;
        for (uint32_t e = lane; e < total; e += 32) {
            int lo = 0, hi = 31;   // owner: largest unit with u_off <= e
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (u_off[warp][mid] <= e) lo = mid; else hi = mid - 1;
            }
            Unit<real> v;
            v.kind = u_kind[warp][lo]; v.cls = u_cls[warp][lo];
            v.ci = u_ci[warp][lo]; v.cj = u_cj[warp][lo]; v.einv = u_einv[warp][lo];
            const uint32_t idx = u_base[warp][lo] + (e - u_off[warp][lo]);
            real ratio, contrib;
            int a, b;
            if (eval_entry<real>(L, V, v, idx, ratio, contrib, a, b)) {
                e_grp += (acc_t)contrib;
                q_grp += rate_of<real>(ratio, &flag);
            }
        }
        e_acc += (double)e_grp;
        q_grp = warp_sum_u128(q_grp);
        if (lane == 0) rates[(size_t)w * n_groups + g] = q_grp;
        q_tot += q_grp;
        __syncwarp();
    }
    e_acc = warp_sum_f64(e_acc);
    if (lane == 0) { red_e[warp] = e_acc; red_q[warp] = q_tot; }
    if (flag) atomicOr(status, flag);
    __syncthreads();
    if (tid == 0) {
        double s = A.e_diag[w];
        u128 Q = 0;
        for (int k = 0; k < VMC_WARPS; ++k) { s += red_e[k]; Q += red_q[k]; }
        e_loc[w] = s;
        if (Q == 0) {
            t_res[w] = 0.0;
            atomicOr(status, VMC_DEV_NOMOVE);
        } else {
            const double qh = (double)(uint64_t)(Q >> 64), ql = (double)(uint64_t)Q;
            t_res[w] = __ddiv_rn(1.0, __dadd_rn(qh, __dmul_rn(ql, 0x1p-64)));
        }
    }
}

// ---------------------------------------------------------------------------------- CTMC
template <typename real>
__global__ void __launch_bounds__(VMC_THREADS)
k_ctmc_step(ListsView L, WalkerArgs A, const double *__restrict__ J, const u128 *__restrict__ rates,
            int n_groups, uint64_t seed, uint64_t *__restrict__ move_code, unsigned *status) {
    const Geo geo = make_geo(A.M, A.na, A.nb);
    const int w = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nt = blockDim.x;
    const int M = geo.M, ne = geo.ne, N2 = 2 * M;
    extern __shared__ __align__(16) unsigned char smraw[];
    uint16_t *pos = (uint16_t *)smraw;
    uint16_t *socc = pos + 2 * M;
    uint16_t *gstart = socc + ne;
    real *vec = (real *)(((uintptr_t)(gstart + ne) + 15) & ~(uintptr_t)15);
    // vec holds: ua[nmax], ub[nmax], gci[M], gcj[M], arow_i[nmax], arow_j[nmax]
    __shared__ int s_move[6];       // kind, i, j, a, b, ok
    __shared__ uint32_t u_off[33];
    __shared__ double red[VMC_WARPS];

    real *Gw = (real *)A.G + (size_t)w * geo.g_stride;
    real *Aw = (real *)A.AinvT + (size_t)w * geo.a_stride;
    real *Sw = (real *)A.S + (size_t)w * N2;
    uint16_t *occ = A.occ_list + (size_t)w * ne;
    uint16_t *virt = A.virt_list + (size_t)w * (2 * M - ne);
    uint32_t *bits = A.occ_bits_w + (size_t)w * 2 * geo.nw;
    build_maps(geo, occ, virt, bits, pos, socc, gstart);
    __syncthreads();

    // ---- choose the group (warp 0), then the entry inside it
    if (warp == 0) {
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
        if (lane == 0) { s_move[0] = 0; s_move[5] = 0; }
        __syncwarp();
        if (gsel >= 0) {
            const u128 Tl = T - before;   // threshold inside the group
            View<real> V;
            V.pos = pos; V.G = Gw; V.E = nullptr; V.S = Sw; V.F = A.F + (size_t)w * 2 * L.ns; V.geo = geo;
            int kg, x, y0;
            decode_group(gsel, ne, gstart, kg, x, y0);
            const int y = y0 + lane;
            Unit<real> u;
            u.base = 0; u.len = 0; u.kind = 0; u.cls = 0; u.ci = 0; u.cj = 0; u.i = 0; u.j = 0;
            u.einv = (real)0;
            if (y < ne) setup_unit<real>(L, V, kg, x, y, socc, u);
            uint32_t inc = u.len;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t o = __shfl_up_sync(0xffffffffu, inc, d);
                if (lane >= d) inc += o;
            }
            u_off[lane] = inc - u.len;
            if (lane == 31) u_off[32] = inc;
            __syncwarp();
            const uint32_t total = u_off[32];
            u128 carry = 0;
            unsigned flag = 0;
            bool found = false;
            for (uint32_t e0 = 0; e0 < total && !found; e0 += 32) {
                const uint32_t e = e0 + lane;
                u128 q = 0;
                int a = -1, b = -1, owner = 0;
                if (e < total) {
                    int lo = 0, hi = 31;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (u_off[mid] <= e) lo = mid; else hi = mid - 1;
                    }
                    owner = lo;
                }
                // fetch the owner's unit fields by shuffles (all lanes participate)
                Unit<real> v;
                v.kind = __shfl_sync(0xffffffffu, u.kind, owner);
                v.cls = __shfl_sync(0xffffffffu, u.cls, owner);
                v.ci = __shfl_sync(0xffffffffu, u.ci, owner);
                v.cj = __shfl_sync(0xffffffffu, u.cj, owner);
                v.einv = __shfl_sync(0xffffffffu, u.einv, owner);
                const uint32_t vbase = __shfl_sync(0xffffffffu, u.base, owner);
                const int vi = __shfl_sync(0xffffffffu, u.i, owner);
                const int vj = __shfl_sync(0xffffffffu, u.j, owner);
                if (e < total) {
                    real ratio, contrib;
                    const uint32_t idx = vbase + (e - u_off[owner]);
                    if (eval_entry<real>(L, V, v, idx, ratio, contrib, a, b)) q = rate_of<real>(ratio, &flag);
                }
                const u128 incl2 = warp_incl_scan_u128(q, lane) + carry;
                const unsigned hit = __ballot_sync(0xffffffffu, e < total && incl2 > Tl);
                if (hit) {
                    const int src = __ffs(hit) - 1;
                    if (lane == src) {
                        s_move[0] = v.kind == 0 ? 1 : 2;
                        s_move[1] = vi; s_move[2] = vj; s_move[3] = a; s_move[4] = b; s_move[5] = 1;
                    }
                    found = true;
                }
                carry = shfl_u128(incl2, 31);
            }
            if (!found && lane == 0) atomicOr(status, VMC_DEV_INCONSISTENT);
        } else if (lane == 0) {
            atomicOr(status, VMC_DEV_NOMOVE);
        }
    }
    __syncthreads();
    const int ok = s_move[5];
    if (!ok) {
        if (tid == 0) { move_code[w] = 0; A.rng[w] += 1; }
        return;
    }
    const int kind = s_move[0], I = s_move[1], Jo = s_move[2], Ao = s_move[3], Bo = s_move[4];
    if (tid == 0) {
        const uint64_t j10 = kind == 2 ? (uint64_t)Jo : 1023ull, b10 = kind == 2 ? (uint64_t)Bo : 1023ull;
        move_code[w] = (uint64_t)kind | ((uint64_t)I << 2) | (j10 << 12) | ((uint64_t)Ao << 22) | (b10 << 32);
    }

    // ---- diagonal energy change (old occupation in socc), FP64
    {
        auto D = [&](int p, int q) -> double {
            const int kp = p % M, kq = q % M;
            double d = L.Jd[(size_t)kp * M + kq];
            if ((p >= M) == (q >= M)) d -= L.Kd[(size_t)kp * M + kq];
            return d;
        };
        double part = 0.0;
        for (int t = tid; t < ne; t += nt) {
            const int K = socc[t];
            if (K != I) part += D(Ao, K) - D(I, K);
            if (kind == 2 && K != I && K != Jo) part += D(Bo, K) - D(Jo, K);
        }
        part = warp_sum_f64(part);
        if (lane == 0) red[warp] = part;
        __syncthreads();
        if (tid == 0) {
            double dE = L.hd[Ao % M] - L.hd[I % M];
            if (kind == 2) dE += L.hd[Bo % M] - L.hd[Jo % M] + D(Bo, Ao) - D(Jo, Ao);
            for (int k = 0; k < VMC_WARPS; ++k) dE += red[k];
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
        double *Fw = A.F + (size_t)w * 2 * L.ns;
        const int nch = kind == 2 ? 4 : 2;
        const int chg[4] = {I, Ao, Jo, Bo};
        for (int64_t e = tid; e < L.ns; e += nt) {
            double f0 = Fw[e], f1 = Fw[L.ns + e];
            for (int c = 0; c < nch; ++c) {
                const int p = chg[c];
                const double sgn = (c & 1) ? 1.0 : -1.0;
                const int t = p >= M, k = p - t * M;
                const double jk = L.Tjk[(size_t)k * L.ns + e], jj = L.Tj[(size_t)k * L.ns + e];
                if (t == 0) { f0 += sgn * jk; f1 += sgn * jj; }
                else { f1 += sgn * jk; f0 += sgn * jj; }
            }
            Fw[e] = f0; Fw[L.ns + e] = f1;
        }
    }
    // ---- determinant tables: rank-1 per spin (singles, opposite-spin doubles) or rank-2
    //      Woodbury (same-spin doubles) on G and AinvT (Sherman-Morrison, Sec. III.B)
    const int nmax = geo.na > geo.nb ? geo.na : geo.nb;
    real *ua = vec, *ub = ua + nmax, *gci = ub + nmax, *gcj = gci + M, *ari = gcj + M, *arj = ari + nmax;
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
    for (int st = 0; st < nsteps; ++st) {
        const int s = sp[st], n = geo.n(s), nv = M - n;
        real *Gs = Gw + geo.g_off(s);
        real *As = Aw + geo.a_off(s);
        uint16_t *occs = occ + (s ? geo.na : 0);
        uint16_t *virts = virt + (s ? geo.nv_a : 0);
        const int ci = pos[s * M + fr[st][0]], sa = pos[s * M + to[st][0]] & 0x7FFF;
        int cj = 0, sb = 0;
        if (rk[st] == 2) { cj = pos[s * M + fr[st][1]]; sb = pos[s * M + to[st][1]] & 0x7FFF; }
        __syncthreads();
        // R = G[(a,b), (ci,cj)], inverse coefficients; ua/ub = R^-1 (G[(a,b),:] - E)
        real r00 = Gs[(size_t)sa * n + ci], r01 = 0, r10 = 0, r11 = 1;
        if (rk[st] == 2) { r01 = Gs[(size_t)sa * n + cj]; r10 = Gs[(size_t)sb * n + ci]; r11 = Gs[(size_t)sb * n + cj]; }
        const real det = r00 * r11 - r01 * r10;
        const real i00 = r11 / det, i01 = -r01 / det, i10 = -r10 / det, i11 = r00 / det;
        for (int c = tid; c < n; c += nt) {
            const real va = Gs[(size_t)sa * n + c] - (c == ci ? (real)1 : (real)0);
            const real vb = rk[st] == 2 ? Gs[(size_t)sb * n + c] - (c == cj ? (real)1 : (real)0) : (real)0;
            ua[c] = i00 * va + i01 * vb;
            ub[c] = i10 * va + i11 * vb;
            ari[c] = As[(size_t)ci * n + c];
            arj[c] = rk[st] == 2 ? As[(size_t)cj * n + c] : (real)0;
        }
        for (int r = tid; r < nv; r += nt) {
            real x = Gs[(size_t)r * n + ci], y = rk[st] == 2 ? Gs[(size_t)r * n + cj] : (real)0;
            if (r == sa) { x = 1; y = 0; }
            if (rk[st] == 2 && r == sb) { x = 0; y = 1; }
            gci[r] = x; gcj[r] = y;
        }
        __syncthreads();
        for (size_t t = tid; t < (size_t)nv * n; t += nt) {
            const int r = (int)(t / n), c = (int)(t % n);
            real old = Gs[t];
            if (r == sa) old = (c == ci) ? (real)1 : (real)0;
            if (rk[st] == 2 && r == sb) old = (c == cj) ? (real)1 : (real)0;
            Gs[t] = old - gci[r] * ua[c] - gcj[r] * ub[c];
        }
        for (size_t t = tid; t < (size_t)n * n; t += nt) {
            const int c = (int)(t / n), x = (int)(t % n);
            As[t] = As[t] - ua[c] * ari[x] - ub[c] * arj[x];
        }
        __syncthreads();
        if (tid == 0) {
            occs[ci] = (uint16_t)to[st][0];
            virts[sa] = (uint16_t)fr[st][0];
            if (rk[st] == 2) { occs[cj] = (uint16_t)to[st][1]; virts[sb] = (uint16_t)fr[st][1]; }
            uint32_t *bw = bits + s * geo.nw;
            for (int k = 0; k < rk[st]; ++k) {
                const int f = fr[st][k], tt = to[st][k];
                bw[f >> 5] &= ~(1u << (f & 31));
                bw[tt >> 5] |= 1u << (tt & 31);
            }
        }
    }
    if (tid == 0) A.rng[w] += 1;
}

}  // namespace

int num_groups(int ne) {
    int g = (ne + 31) / 32;
    for (int x = 0; x + 1 < ne; ++x) g += chunks_of_row(ne, x);
    return g;
}

static WalkerArgs make_args(vmc_walkers *Wk) {
    WalkerArgs A;
    A.W = Wk->W; A.M = Wk->M; A.na = Wk->n_alpha; A.nb = Wk->n_beta;
    A.occ_bits = Wk->occ_bits; A.occ_bits_w = Wk->occ_bits;
    A.occ_list = Wk->occ_list; A.virt_list = Wk->virt_list;
    A.G = Wk->G; A.AinvT = Wk->AinvT; A.S = Wk->S; A.F = Wk->F; A.e_diag = Wk->e_diag;
    A.rng = Wk->rng_counter;
    return A;
}

vmc_status launch_local_energy(vmc_ctx *ctx, const vmc_lists *L, vmc_walkers *Wk, double *e_loc,
                               double *t_res, u128 *rates, int n_groups) {
    const int M = Wk->M, ne = Wk->n_alpha + Wk->n_beta;
    const size_t esz = Wk->precision == VMC_FP64 ? 8 : 4;
    const size_t gst = walker_stride_G(M, Wk->n_alpha, Wk->n_beta);
    const size_t smem = esz * (gst + 2 * (size_t)M) + 2 * (2 * (size_t)M + 2 * (size_t)ne) + 16;
    if (smem > 200 * 1024) return set_err(ctx, VMC_ERR_ARG, "walker G table does not fit in shared memory");
    WalkerArgs A = make_args(Wk);
    cudaError_t e;
    if (Wk->precision == VMC_FP64) {
        e = cudaFuncSetAttribute(k_local_energy<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            k_local_energy<double><<<Wk->W, VMC_THREADS, smem, ctx->stream>>>(L->view, A, e_loc, t_res, rates,
                                                                              n_groups, ctx->d_status);
    } else {
        e = cudaFuncSetAttribute(k_local_energy<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            k_local_energy<float><<<Wk->W, VMC_THREADS, smem, ctx->stream>>>(L->view, A, e_loc, t_res, rates,
                                                                             n_groups, ctx->d_status);
    }
    ctx->launches += 1;
    if (e == cudaSuccess) e = cudaGetLastError();
    return cuda_check(ctx, e, "k_local_energy");
}

vmc_status launch_ctmc_step(vmc_ctx *ctx, const vmc_lists *L, const vmc_params *P, vmc_walkers *Wk,
                            uint64_t seed, const u128 *rates, int n_groups, uint64_t *move_code) {
    const int M = Wk->M, ne = Wk->n_alpha + Wk->n_beta;
    const int nmax = Wk->n_alpha > Wk->n_beta ? Wk->n_alpha : Wk->n_beta;
    const size_t esz = Wk->precision == VMC_FP64 ? 8 : 4;
    const size_t smem = 2 * (2 * (size_t)M + 2 * (size_t)ne) + 32 + esz * (4 * (size_t)nmax + 2 * (size_t)M);
    WalkerArgs A = make_args(Wk);
    cudaError_t e;
    if (Wk->precision == VMC_FP64) {
        e = cudaFuncSetAttribute(k_ctmc_step<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            k_ctmc_step<double><<<Wk->W, VMC_THREADS, smem, ctx->stream>>>(L->view, A, P->J, rates, n_groups, seed,
                                                                           move_code, ctx->d_status);
    } else {
        e = cudaFuncSetAttribute(k_ctmc_step<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            k_ctmc_step<float><<<Wk->W, VMC_THREADS, smem, ctx->stream>>>(L->view, A, P->J, rates, n_groups, seed,
                                                                          move_code, ctx->d_status);
    }
    ctx->launches += 1;
    if (e == cudaSuccess) e = cudaGetLastError();
    return cuda_check(ctx, e, "k_ctmc_step");
}
