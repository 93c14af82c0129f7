// Walker tables (Sec. III.B): the one O(N^3) inverse per determinant and the O(1)-ratio tables
// built from it -- G = C C_occ^-1 (Eq. R), the Jastrow sums, the single-excitation Fock sums
// and the diagonal energy.  Also ln|psi| per walker (forward of the ln psi autograd function).
#include <math.h>

#include "common.cuh"

namespace {

// Gauss-Jordan elimination with partial pivoting (an LU factorisation whose inverse is
// accumulated in place) of the n x n FP64 matrix B held in shared memory with row stride ld.
// X (same layout) receives B^-1.  Returns (in *sing) whether a zero pivot was met.
__device__ void gj_invert(double *B, double *X, int n, int ld, double *colk, int *s_piv,
                          int *sing) {
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
    for (int t = tid; t < n * ld; t += nt) X[t] = 0.0;
    __syncthreads();
    for (int r = tid; r < n; r += nt) X[r * ld + r] = 1.0;
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        if (warp == 0) {
            double best = -1.0;
            int idx = k;
            for (int r = k + lane; r < n; r += 32) {
                const double v = fabs(B[r * ld + k]);
                if (v > best) { best = v; idx = r; }
            }
#pragma unroll
            for (int m = 16; m >= 1; m >>= 1) {
                const double ob = __shfl_xor_sync(0xffffffffu, best, m);
                const int oi = __shfl_xor_sync(0xffffffffu, idx, m);
                if (ob > best || (ob == best && oi < idx)) { best = ob; idx = oi; }
            }
            if (lane == 0) *s_piv = idx;
        }
        __syncthreads();
        const int p = *s_piv;
        if (p != k) {
            for (int c = tid; c < 2 * n; c += nt) {
                double *A = c < n ? B : X;
                const int cc = c < n ? c : c - n;
                const double t = A[k * ld + cc];
                A[k * ld + cc] = A[p * ld + cc];
                A[p * ld + cc] = t;
            }
        }
        __syncthreads();
        double d = B[k * ld + k];
        if (d == 0.0) {
            if (tid == 0) *sing = 1;
            d = 1.0;
        }
        __syncthreads();
        for (int c = tid; c < 2 * n; c += nt) {
            if (c < n) B[k * ld + c] = B[k * ld + c] / d;
            else X[k * ld + (c - n)] = X[k * ld + (c - n)] / d;
        }
        for (int r = tid; r < n; r += nt) colk[r] = B[r * ld + k];
        __syncthreads();
        for (int r = warp; r < n; r += (nt >> 5)) {     // rows over warps, columns over lanes
            if (r == k) continue;
            const double f = colk[r];
            for (int c = lane; c < n; c += 32) {
                B[r * ld + c] -= f * B[k * ld + c];
                X[r * ld + c] -= f * X[k * ld + c];
            }
        }
        __syncthreads();
    }
}

// LU with partial pivoting in shared memory; returns log|det| and sign (0 if singular).
__device__ void lu_logdet(double *B, int n, int ld, int *s_piv, double *s_acc, double *logabs,
                          int *sign) {
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
    __shared__ double s_log;
    __shared__ int s_sgn;
    if (tid == 0) { s_log = 0.0; s_sgn = 1; }
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        if (warp == 0) {
            double best = -1.0;
            int idx = k;
            for (int r = k + lane; r < n; r += 32) {
                const double v = fabs(B[r * ld + k]);
                if (v > best) { best = v; idx = r; }
            }
#pragma unroll
            for (int m = 16; m >= 1; m >>= 1) {
                const double ob = __shfl_xor_sync(0xffffffffu, best, m);
                const int oi = __shfl_xor_sync(0xffffffffu, idx, m);
                if (ob > best || (ob == best && oi < idx)) { best = ob; idx = oi; }
            }
            if (lane == 0) *s_piv = idx;
        }
        __syncthreads();
        const int p = *s_piv;
        if (p != k) {
            for (int c = tid; c < n; c += nt) {
                const double t = B[k * ld + c];
                B[k * ld + c] = B[p * ld + c];
                B[p * ld + c] = t;
            }
        }
        __syncthreads();
        const double d = B[k * ld + k];
        if (tid == 0) {
            if (p != k) s_sgn = -s_sgn;
            if (d == 0.0) s_sgn = 0;
            else {
                s_log += log(fabs(d));
                if (d < 0) s_sgn = -s_sgn;
            }
        }
        for (int t = tid; t < (n - k - 1) * (n - k); t += nt) {
            const int r = k + 1 + t / (n - k), c = k + t % (n - k);
            if (c == k) continue;
            const double f = B[r * ld + k] / (d == 0.0 ? 1.0 : d);
            B[r * ld + c] -= f * B[k * ld + c];
        }
        __syncthreads();
    }
    (void)s_acc;
    *logabs = s_log;
    *sign = s_sgn;
}

template <typename real>
__global__ void __launch_bounds__(VMC_THREADS)
k_init_tables(int M, int na, int nb, const double *__restrict__ Ca, const double *__restrict__ Cb,
              uint16_t *occ_list, uint16_t *virt_list, uint16_t *pos_all, uint32_t *occ_bits, real *G,
              real *AinvT, unsigned *status) {
    const int w = blockIdx.x, sg = blockIdx.y;
    const int n = sg ? nb : na, nv = M - n;
    const int ne = na + nb, nw = (M + 31) / 32;
    const double *C = sg ? Cb : Ca;
    const int tid = threadIdx.x, nt = blockDim.x;
    extern __shared__ double sm[];
    const int ld = n + 1;
    double *B = sm;
    double *X = B + (size_t)n * ld;
    double *colk = X + (size_t)n * ld;
    __shared__ uint16_t s_occ[VMC_MAX_M], s_virt[VMC_MAX_M];
    __shared__ uint8_t mark[VMC_MAX_M];
    __shared__ int s_piv, s_sing;
    const uint16_t *occ = occ_list + (size_t)w * ne + (sg ? na : 0);
    uint16_t *vl = virt_list + (size_t)w * (2 * M - ne) + (sg ? M - na : 0);
    for (int k = tid; k < M; k += nt) mark[k] = 0;
    if (tid == 0) s_sing = 0;
    __syncthreads();
    for (int c = tid; c < n; c += nt) {
        s_occ[c] = occ[c];
        mark[occ[c]] = 1;
    }
    __syncthreads();
    if (tid == 0) {   // virtual slots: unoccupied orbitals ascending
        int v = 0;
        for (int k = 0; k < M; ++k)
            if (!mark[k]) s_virt[v++] = (uint16_t)k;
    }
    for (int q = tid; q < nw; q += nt) {
        uint32_t word = 0;
        for (int b = 0; b < 32; ++b) {
            const int k = q * 32 + b;
            if (k < M && mark[k]) word |= 1u << b;
        }
        occ_bits[((size_t)w * 2 + sg) * nw + q] = word;
    }
    // B = C_occ^T: B[x][c] = C[occ[c]][x]
    for (int t = tid; t < n * n; t += nt) {
        const int x = t / n, c = t % n;
        B[x * ld + c] = C[(size_t)s_occ[c] * n + x];
    }
    __syncthreads();
    {
        uint16_t *pw = pos_all + (size_t)w * 2 * M + (size_t)sg * M;
        for (int s = tid; s < nv; s += nt) {
            vl[s] = s_virt[s];
            pw[s_virt[s]] = (uint16_t)(0x8000 | s);
        }
        for (int c = tid; c < n; c += nt) pw[s_occ[c]] = (uint16_t)c;
    }
    if (n > 0) gj_invert(B, X, n, ld, colk, &s_piv, &s_sing);   // X = (C_occ^T)^-1 = AinvT
    __syncthreads();
    if (s_sing && tid == 0) atomicOr(status, VMC_DEV_SINGULAR);
    const size_t gofs = (size_t)w * ((size_t)(M - na) * na + (size_t)(M - nb) * nb) +
                        (sg ? (size_t)(M - na) * na : 0);
    const size_t aofs = (size_t)w * ((size_t)na * na + (size_t)nb * nb) + (sg ? (size_t)na * na : 0);
    for (int t = tid; t < n * n; t += nt) {
        const int c = t / n, x = t % n;
        AinvT[aofs + t] = (real)X[c * ld + x];
    }
    // G[s][c] = sum_x C[virt[s]][x] Ainv[x][c] = sum_x C[virt[s]][x] AinvT[c][x]
    for (int t = tid; t < nv * n; t += nt) {
        const int s = t / n, c = t % n;
        const double *crow = C + (size_t)s_virt[s] * n;
        double acc = 0.0;
        for (int x = 0; x < n; ++x) acc += crow[x] * X[c * ld + x];
        G[gofs + t] = (real)acc;
    }
}

__device__ void refresh_orbitals(int w, int sg, int M, int na, int nb, const uint16_t *occ_list,
                                 uint16_t *virt_list, uint16_t *pos_all, uint32_t *occ_bits, uint16_t *s_occ,
                                 uint16_t *s_virt, uint8_t *mark);

// Mixed form: LU of C_occ^T with partial pivoting in FP64 (in shared memory), then the inverse
// from the factors and G = C C_occ^-1 in FP32, the precision these tables are kept in.
// Shared memory: one n x (n+1) FP64 buffer; after the factorisation it is reused as two FP32
// n x (n+1) arrays (factors, inverse), so four CTAs fit on an SM.
__global__ void __launch_bounds__(VMC_THREADS)
k_init_tables_mixed(int M, int na, int nb, const double *__restrict__ Ca, const double *__restrict__ Cb,
                    const float *__restrict__ Cf, uint16_t *occ_list, uint16_t *virt_list, uint16_t *pos_all,
                    uint32_t *occ_bits, float *G, float *AinvT, unsigned *status, int do_g) {
    const int w = blockIdx.x, sg = blockIdx.y;
    const int n = sg ? nb : na, nv = M - n;
    const int ne = na + nb, nw = (M + 31) / 32;
    const double *C = sg ? Cb : Ca;
    const float *Csf = Cf + (sg ? (size_t)M * na : 0);     // FP32 copy of C^sigma
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
    extern __shared__ double sm[];
    const int ld = n + 1;
    double *B = sm;                               // n x ld FP64: LU factors
    float *LUf = (float *)sm;                     // n x ld FP32 (aliases B after the factorisation)
    float *Y = LUf + (size_t)n * ld;              // n x ld FP32
    __shared__ uint16_t s_occ[VMC_MAX_M], s_virt[VMC_MAX_M];
    __shared__ uint8_t mark[VMC_MAX_M];
    __shared__ int perm[VMC_MAX_M];
    __shared__ int s_sing;
    (void)ne; (void)nw; (void)nv;
    if (tid == 0) s_sing = 0;
    // occupied/virtual lists, occupation words and the orbital map (ends with a barrier after s_occ)
    refresh_orbitals(w, sg, M, na, nb, occ_list, virt_list, pos_all, occ_bits, s_occ, s_virt, mark);
    for (int c = tid; c < n; c += nt) perm[c] = c;
    for (int t = tid; t < n * n; t += nt) {       // B = C_occ^T: B[x][c] = C[occ[c]][x], read along rows of C
        const int c = t / n, x = t % n;
        B[x * ld + c] = C[(size_t)s_occ[c] * n + x];
    }
    __syncthreads();
    // ---- LU with partial pivoting, FP64: P B = L U, rows left in place (row list rl: rl[k] = the
    //      row that is pivot k).  Look-ahead: while warps 1.. update columns k+2.. of step k, warp 0
    //      updates column k+1, picks the pivot of step k+1 into the other row list and scales its
    //      multipliers, so the serial pivot work overlaps the FP64 update.
    __shared__ int perm2[VMC_MAX_M];
    auto pivot = [&](int k, const int *rin, int *rout) {      // warp 0 only
        for (int r = lane; r < n; r += 32) rout[r] = rin[r];
        __syncwarp();
        // partial pivoting on |B[r][k]|, compared as the integer bits of |v| plus one (0: NaN or no
        // row), so the warp reductions run on the integer pipe; ties go to the lowest row
        unsigned long long best = 0ull;
        int idx = k;
        for (int r = k + lane; r < n; r += 32) {
            const unsigned long long a =
                (unsigned long long)__double_as_longlong(B[rout[r] * ld + k]) & 0x7FFFFFFFFFFFFFFFull;
            const unsigned long long key = a > 0x7FF0000000000000ull ? 0ull : a + 1ull;
            if (key > best) { best = key; idx = r; }
        }
        const uint32_t bh = (uint32_t)(best >> 32), bl = (uint32_t)best;
        const uint32_t mh = __reduce_max_sync(0xffffffffu, bh);
        const uint32_t ml = __reduce_max_sync(0xffffffffu, bh == mh ? bl : 0u);
        idx = __reduce_min_sync(0xffffffffu, (bh == mh && bl == ml) ? idx : 0x7FFFFFFF);
        if (lane == 0 && idx != k) { const int t = rout[k]; rout[k] = rout[idx]; rout[idx] = t; }
        __syncwarp();
        const double d = B[rout[k] * ld + k];
        const bool zero = ((unsigned long long)__double_as_longlong(d) << 1) == 0ull;   // +-0
        if (zero && lane == 0) s_sing = 1;
        const double dinv = zero ? 1.0 : __drcp_rn(d);
        for (int r = k + 1 + lane; r < n; r += 32) B[rout[r] * ld + k] *= dinv;
    };
    if (n > 0 && warp == 0) pivot(0, perm, perm2);
    __syncthreads();
    int *cur = perm2, *nxt = perm;
    for (int k = 0; k + 1 < n; ++k) {
        const double *rowk = B + cur[k] * ld;
        if (warp == 0) {
            for (int r = k + 1 + lane; r < n; r += 32) {
                double *row = B + cur[r] * ld;
                row[k + 1] = fma(-row[k], rowk[k + 1], row[k + 1]);
            }
            __syncwarp();
            pivot(k + 1, cur, nxt);
        } else {
            // B[r][c] -= B[r][k] B[pivot k][c] for the unused rows r and c >= k+2, flattened over
            // warps 1.. so that every lane has an element (the FP64 pipe is the bound here)
            const int wr = n - k - 1, wc = n - k - 2, tot = wr * wc, t0 = tid - 32, nth = nt - 32;
            if (wc > 0 && t0 < tot) {
                const int sr = nth / wc, sc = nth - sr * wc;   // advance of the flat index by nth
                int rr = t0 / wc, cc = t0 - rr * wc;
                for (int t = t0; t < tot; t += nth) {
                    double *row = B + cur[k + 1 + rr] * ld;
                    row[k + 2 + cc] = fma(-row[k], rowk[k + 2 + cc], row[k + 2 + cc]);
                    cc += sc; rr += sr;
                    if (cc >= wc) { cc -= wc; ++rr; }
                }
            }
        }
        __syncthreads();
        int *t = cur; cur = nxt; nxt = t;
    }
    const int *rl = cur;
    if (s_sing && tid == 0) atomicOr(status, VMC_DEV_SINGULAR);
    // reciprocals of U's diagonal (one FP64 division per row, not per element; n <= 128)
    __shared__ double rdiag[VMC_MAX_M / 2];
    for (int r = tid; r < n; r += nt) rdiag[r] = __drcp_rn(B[rl[r] * ld + r]);
    __syncthreads();
    // ---- FP32 copies: unit-lower L, unit-upper U' = D^-1 U, and 1/D; the buffer is reused
    {
        const int per = (n * n + nt - 1) / nt;
        float vals[(VMC_MAX_M / 2 + 1) * (VMC_MAX_M / 2 + 1) / VMC_THREADS + 2];
        int cnt = 0;
        for (int t = tid; t < n * n && cnt < per; t += nt, ++cnt) {
            const int r = t / n, c = t % n;
            const double v = B[rl[r] * ld + c];
            vals[cnt] = c > r ? (float)(v * rdiag[r]) : (c == r ? (float)rdiag[r] : (float)v);
        }
        __syncthreads();
        cnt = 0;
        for (int t = tid; t < n * n && cnt < per; t += nt, ++cnt) {
            const int r = t / n, c = t % n;
            LUf[r * ld + c] = vals[cnt];
            Y[r * ld + c] = rl[r] == c ? 1.0f : 0.0f;        // rows of the permutation
        }
        __syncthreads();
    }
    // ---- Y <- U'^-1 D^-1 L^-1 Y by blocked substitution: per block of kSB pivot rows every warp
    //      solves the block for its lanes' columns in registers (redundantly, a few FMAs), then
    //      updates its share of the other rows with all kSB pivot rows at once; one barrier per
    //      block.  The finished block rows are stored after the barrier (no warp reads them again).
    const int nwarp = nt >> 5;
    constexpr int kSB = 4, kCL = (VMC_MAX_M / 2 + 31) / 32;   // pivot rows per block, columns per lane
    for (int k0 = 0; k0 < n; k0 += kSB) {          // forward: L (unit diagonal)
        const int kb = min(kSB, n - k0);
        float yh[kSB][kCL];
#pragma unroll
        for (int t = 0; t < kSB; ++t)
#pragma unroll
            for (int i = 0; i < kCL; ++i) {
                const int c = lane + 32 * i;
                yh[t][i] = (t < kb && c < n) ? Y[(k0 + t) * ld + c] : 0.0f;
            }
#pragma unroll
        for (int t = 1; t < kSB; ++t)
#pragma unroll
            for (int q = 0; q < kSB - 1; ++q)
                if (q < t && t < kb) {
                    const float l = LUf[(k0 + t) * ld + k0 + q];
#pragma unroll
                    for (int i = 0; i < kCL; ++i) yh[t][i] -= l * yh[q][i];
                }
        for (int r = k0 + kb + warp; r < n; r += nwarp) {
            float l[kSB];
#pragma unroll
            for (int t = 0; t < kSB; ++t) l[t] = t < kb ? LUf[r * ld + k0 + t] : 0.0f;
#pragma unroll
            for (int i = 0; i < kCL; ++i) {
                const int c = lane + 32 * i;
                if (c < n) {
                    float v = Y[r * ld + c];
#pragma unroll
                    for (int t = 0; t < kSB; ++t) v -= l[t] * yh[t][i];
                    Y[r * ld + c] = v;
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int t = 1; t < kSB; ++t)
            if (t < kb && warp == (t - 1) % nwarp)
#pragma unroll
                for (int i = 0; i < kCL; ++i) {
                    const int c = lane + 32 * i;
                    if (c < n) Y[(k0 + t) * ld + c] = yh[t][i];
                }
    }
    __syncthreads();
    for (int r = warp; r < n; r += nwarp) {       // D^-1
        const float d = LUf[r * ld + r];
        for (int c = lane; c < n; c += 32) Y[r * ld + c] *= d;
    }
    __syncthreads();
    for (int k1 = n - 1; k1 >= 0; k1 -= kSB) {     // backward: U' (unit diagonal), blocks from the bottom
        const int kb = min(kSB, k1 + 1), p0 = k1 - kb + 1;   // block rows p0 .. k1
        float yh[kSB][kCL];
#pragma unroll
        for (int t = 0; t < kSB; ++t)
#pragma unroll
            for (int i = 0; i < kCL; ++i) {
                const int c = lane + 32 * i;
                yh[t][i] = (t < kb && c < n) ? Y[(p0 + t) * ld + c] : 0.0f;
            }
#pragma unroll
        for (int t = kSB - 2; t >= 0; --t)
#pragma unroll
            for (int q = 1; q < kSB; ++q)
                if (q > t && q < kb) {
                    const float u = LUf[(p0 + t) * ld + p0 + q];
#pragma unroll
                    for (int i = 0; i < kCL; ++i) yh[t][i] -= u * yh[q][i];
                }
        for (int r = warp; r < p0; r += nwarp) {
            float u[kSB];
#pragma unroll
            for (int t = 0; t < kSB; ++t) u[t] = t < kb ? LUf[r * ld + p0 + t] : 0.0f;
#pragma unroll
            for (int i = 0; i < kCL; ++i) {
                const int c = lane + 32 * i;
                if (c < n) {
                    float v = Y[r * ld + c];
#pragma unroll
                    for (int t = 0; t < kSB; ++t) v -= u[t] * yh[t][i];
                    Y[r * ld + c] = v;
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int t = 0; t < kSB - 1; ++t)
            if (t < kb - 1 && warp == t % nwarp)
#pragma unroll
                for (int i = 0; i < kCL; ++i) {
                    const int c = lane + 32 * i;
                    if (c < n) Y[(p0 + t) * ld + c] = yh[t][i];
                }
    }
    __syncthreads();
    // Y = B^-1 = (C_occ^T)^-1 = AinvT
    const size_t gofs = (size_t)w * ((size_t)(M - na) * na + (size_t)(M - nb) * nb) +
                        (sg ? (size_t)(M - na) * na : 0);
    const size_t aofs = (size_t)w * ((size_t)na * na + (size_t)nb * nb) + (sg ? (size_t)na * na : 0);
    for (int t = tid; t < n * n; t += nt) {
        const int c = t / n, x = t % n;
        AinvT[aofs + t] = Y[c * ld + x];
    }
    if (!do_g) return;   // G is formed on the tensor cores by k_g_umma
    // G[s][c] = sum_x C[virt[s]][x] AinvT[c][x]: 4 x 4 register tiles (slots x columns)
    const int ts = (nv + 3) / 4, tc = (n + 3) / 4;
    for (int tile = tid; tile < ts * tc; tile += nt) {
        const int s0 = (tile / tc) * 4, c0 = (tile % tc) * 4;
        float acc[4][4] = {};
        const float *cr[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) cr[i] = Csf + (size_t)s_virt[min(s0 + i, nv - 1)] * n;
        for (int x = 0; x < n; ++x) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = __ldg(cr[i] + x);
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Y[min(c0 + j, n - 1) * ld + x];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (s0 + i < nv && c0 + j < n) G[gofs + (size_t)(s0 + i) * n + c0 + j] = acc[i][j];
    }
}

// Mixed form: the Fock sums F[s][e] = h_ai + sum_k n_k^s Tjk[k][e] + n_k^(1-s) Tj[k][e] in FP32 for
// kFockWalkers walkers per CTA (each table row is read once per CTA), one singles entry per thread;
// rewritten at every refresh so that the per-move FP32 updates never accumulate beyond one period.
constexpr int kFockWalkers = 16, kFockThreads = 128;

__global__ void __launch_bounds__(kFockThreads)
k_fock_sums_f32(ListsView L, int W, const uint32_t *__restrict__ occ_bits, float *F) {
    const int M = L.M, nw = (M + 31) / 32, w0 = blockIdx.y * kFockWalkers;
    __shared__ float2 occf[VMC_MAX_M][kFockWalkers];   // (n_alpha, n_beta) of orbital k per walker
    for (int t = threadIdx.x; t < M * kFockWalkers; t += blockDim.x) {
        const int k = t / kFockWalkers, q = t % kFockWalkers, w = w0 + q;
        float2 o = make_float2(0.f, 0.f);
        if (w < W) {
            const uint32_t *b = occ_bits + (size_t)w * 2 * nw;
            o.x = (float)((b[k >> 5] >> (k & 31)) & 1u);
            o.y = (float)((b[nw + (k >> 5)] >> (k & 31)) & 1u);
        }
        occf[k][q] = o;
    }
    __syncthreads();
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= L.ns_pad) return;
    const int64_t np = L.ns_pad;
    float acc[kFockWalkers][2];
    const float h = e < L.ns ? (float)L.h1[(size_t)L.s_a[e] * M + L.s_owner[e]] : 0.f;
#pragma unroll
    for (int q = 0; q < kFockWalkers; ++q) acc[q][0] = acc[q][1] = h;
    for (int k = 0; k < M; ++k) {
        const float tk = __ldg(L.Tjkf + (size_t)k * np + e), tx = __ldg(L.Tjf + (size_t)k * np + e);
#pragma unroll
        for (int q = 0; q < kFockWalkers; ++q) {
            const float2 o = occf[k][q];
            acc[q][0] = fmaf(o.x, tk, fmaf(o.y, tx, acc[q][0]));
            acc[q][1] = fmaf(o.y, tk, fmaf(o.x, tx, acc[q][1]));
        }
    }
#pragma unroll
    for (int q = 0; q < kFockWalkers; ++q)
        if (w0 + q < W) {
            F[((size_t)(w0 + q) * 2) * np + e] = acc[q][0];
            F[((size_t)(w0 + q) * 2 + 1) * np + e] = acc[q][1];
        }
}

// ---- Register-resident Gauss-Jordan refresh (both forms) ---------------------------------------
// One CTA of kGJ x kGJ threads per (walker, spin).  Thread (ty, tx) keeps B[r][c] for r = ty + kGJ i,
// c = tx + kGJ j (i, j < R) in registers; a half-warp shares tx, so the threads owning a column are
// one half-warp and find its pivot with shuffles.  In-place elimination with implicit row pivoting:
// step k picks the unused row p with the largest |B[p][k]|, scales row p by d = 1/B[p][k] (its k-th
// entry becoming d), and subtracts B[r][k] times that row from every other row r (their k-th entry
// becoming -B[r][k] d).  That is n^3 multiply-adds, two barriers per step, and no row exchanges; the
// result X satisfies B^-1[k][piv[j]] = X[piv[k]][j].
constexpr int kGJ = 16;
constexpr int kNoRow = 0x7fffffff;

// Orbital bookkeeping shared by the refresh kernels: occupied/virtual lists of spin sg, its
// occupation bits and the orbital -> column/slot map.
__device__ void refresh_orbitals(int w, int sg, int M, int na, int nb, const uint16_t *occ_list,
                                 uint16_t *virt_list, uint16_t *pos_all, uint32_t *occ_bits, uint16_t *s_occ,
                                 uint16_t *s_virt, uint8_t *mark) {
    const int n = sg ? nb : na, nv = M - n, ne = na + nb, nw = (M + 31) / 32;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const uint16_t *occ = occ_list + (size_t)w * ne + (sg ? na : 0);
    for (int k = tid; k < M; k += nt) mark[k] = 0;
    __syncthreads();
    for (int c = tid; c < n; c += nt) {
        s_occ[c] = occ[c];
        mark[occ[c]] = 1;
    }
    __syncthreads();
    if (warp == 0) {   // virtual slots: unoccupied orbitals ascending; occupation words
        int v = 0;
        for (int b0 = 0; b0 < M; b0 += 32) {
            const int k = b0 + lane;
            const bool occd = k < M && mark[k];
            const unsigned bal = __ballot_sync(0xffffffffu, k < M && !occd);
            if (k < M && !occd) s_virt[v + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)k;
            v += __popc(bal);
            const unsigned word = __ballot_sync(0xffffffffu, occd);
            if (lane == 0) occ_bits[((size_t)w * 2 + sg) * nw + (b0 >> 5)] = word;
        }
    }
    __syncthreads();
    uint16_t *vl = virt_list + (size_t)w * (2 * M - ne) + (sg ? M - na : 0);
    uint16_t *pw = pos_all + (size_t)w * 2 * M + (size_t)sg * M;
    for (int s = tid; s < nv; s += nt) {
        vl[s] = s_virt[s];
        pw[s_virt[s]] = (uint16_t)(0x8000 | s);
    }
    for (int c = tid; c < n; c += nt) pw[s_occ[c]] = (uint16_t)c;
}

__device__ __forceinline__ unsigned long long abs_bits(double v) {
    return (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
}
__device__ __forceinline__ unsigned long long abs_bits(float v) { return __float_as_uint(v) & 0x7FFFFFFFu; }
__device__ __forceinline__ unsigned long long abs_inf_bits(double) { return 0x7FF0000000000000ull; }
__device__ __forceinline__ unsigned long long abs_inf_bits(float) { return 0x7F800000ull; }
__device__ __forceinline__ double rcp_rn(double d) { return __drcp_rn(d); }
__device__ __forceinline__ float rcp_rn(float d) { return __frcp_rn(d); }

template <typename real, int R>
__global__ void __launch_bounds__(kGJ * kGJ, sizeof(real) == 4 ? (R <= 5 ? 4 : 2) : (R <= 5 ? 3 : 1))
k_refresh_gj(int M, int na, int nb, const real *__restrict__ Ca, const real *__restrict__ Cb,
             const uint16_t *occ_list, uint16_t *virt_list, uint16_t *pos_all, uint32_t *occ_bits, real *G,
             real *AinvT, unsigned *status, int do_g) {
    constexpr int NR = kGJ * R;
    const int w = blockIdx.x, sg = blockIdx.y;
    const int n = sg ? nb : na, nv = M - n, ld = n + 1;
    const real *C = sg ? Cb : Ca;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int tx = tid >> 4, ty = tid & 15;
    extern __shared__ __align__(16) unsigned char gj_smem[];
    real *Y = (real *)gj_smem;                       // n x ld: the inverse (C_occ^T)^-1 = AinvT
    __shared__ real pcol[2][NR], prow[2][NR], s_d[2];
    __shared__ int s_p[2], piv[NR], rstep[NR], s_sing;
    __shared__ uint16_t s_occ[VMC_MAX_M], s_virt[VMC_MAX_M];
    __shared__ uint8_t mark[VMC_MAX_M];
    if (tid == 0) s_sing = 0;
    refresh_orbitals(w, sg, M, na, nb, occ_list, virt_list, pos_all, occ_bits, s_occ, s_virt, mark);
    __syncthreads();
    // B = C_occ^T: B[r][c] = C[occ[c]][r]; a half-warp reads 16 consecutive r of one orbital row
    real X[R][R];
    unsigned used = 0;
#pragma unroll
    for (int i = 0; i < R; ++i)
        if (ty + kGJ * i >= n) used |= 1u << i;
#pragma unroll
    for (int j = 0; j < R; ++j) {
        const int c = tx + kGJ * j;
        const real *crow = C + (size_t)(c < n ? s_occ[c] : 0) * n;
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const int r = ty + kGJ * i;
            X[i][j] = (r < n && c < n) ? crow[r] : real(0);
        }
    }
    const unsigned hmask = 0xFFFFu << ((tx & 1) * 16);
    for (int k = 0; k < n; ++k) {
        const int b = k & 1, kj = k >> 4;
        if (tx == (k & 15)) {                        // pivot search in column k (one half-warp)
            // candidates: the unused rows; key = |v| bits + 2 (1 for NaN), compared as integers so
            // the half-warp reductions run on the integer pipe; ties go to the lowest row
            unsigned long long best = 0ull;
            int bi = kNoRow;
#pragma unroll
            for (int i = 0; i < R; ++i) {
                real v = real(0);
#pragma unroll
                for (int j = 0; j < R; ++j)
                    if (j == kj) v = X[i][j];
                const int r = ty + kGJ * i;
                if (r < n) pcol[b][r] = v;
                const unsigned long long a = abs_bits(v);
                const unsigned long long key = a > abs_inf_bits(v) ? 1ull : a + 2ull;
                if (!((used >> i) & 1u) && key > best) { best = key; bi = r; }
            }
            const uint32_t bh = (uint32_t)(best >> 32), bl = (uint32_t)best;
            const uint32_t mh = __reduce_max_sync(hmask, bh);
            const uint32_t ml = __reduce_max_sync(hmask, bh == mh ? bl : 0u);
            bi = __reduce_min_sync(hmask, (bh == mh && bl == ml) ? bi : 0x7FFFFFFF);
            __syncwarp(hmask);
            if (ty == 0) {
                real d = pcol[b][bi];
                if (d == real(0) || !isfinite(d)) { s_sing = 1; d = real(1); }
                s_p[b] = bi;
                s_d[b] = rcp_rn(d);
                piv[k] = bi;
                rstep[bi] = k;
            }
        }
        __syncthreads();
        const int p = s_p[b], pi = p >> 4;
        const real d = s_d[b];
        const bool prow_owner = ty == (p & 15), kcol_owner = tx == (k & 15);
        if (prow_owner) {                            // the pivot row, scaled (its k-th entry: d)
            used |= 1u << pi;
#pragma unroll
            for (int i = 0; i < R; ++i)
                if (i == pi) {
#pragma unroll
                    for (int j = 0; j < R; ++j) {
                        const int c = tx + kGJ * j;
                        const real val = c == k ? d : X[i][j] * d;
                        X[i][j] = val;
                        if (c < n) prow[b][c] = val;
                    }
                }
        }
        __syncthreads();
        // every other row: X[r][c] -= B[r][k] prow[c]; then the column-k owners set X[r][k] = -B[r][k] d
        real pr[R], f[R];
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const int c = tx + kGJ * j;
            pr[j] = c < n ? prow[b][c] : real(0);
        }
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const int r = ty + kGJ * i;
            f[i] = (r < n && r != p) ? pcol[b][r] : real(0);
        }
#pragma unroll
        for (int i = 0; i < R; ++i)
#pragma unroll
            for (int j = 0; j < R; ++j) X[i][j] = fma(-f[i], pr[j], X[i][j]);
        if (kcol_owner) {
#pragma unroll
            for (int i = 0; i < R; ++i)
                if (ty + kGJ * i != p) {
#pragma unroll
                    for (int j = 0; j < R; ++j)
                        if (j == kj) X[i][j] = -f[i] * d;
                }
        }
    }
    __syncthreads();
    if (s_sing && tid == 0) atomicOr(status, VMC_DEV_SINGULAR);
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int r = ty + kGJ * i;
        if (r < n) {
            const int yr = rstep[r] * ld;
#pragma unroll
            for (int j = 0; j < R; ++j) {
                const int c = tx + kGJ * j;
                if (c < n) Y[yr + piv[c]] = X[i][j];
            }
        }
    }
    __syncthreads();
    const size_t gofs = (size_t)w * ((size_t)(M - na) * na + (size_t)(M - nb) * nb) +
                        (sg ? (size_t)(M - na) * na : 0);
    const size_t aofs = (size_t)w * ((size_t)na * na + (size_t)nb * nb) + (sg ? (size_t)na * na : 0);
    for (int t = tid; t < n * n; t += nt) AinvT[aofs + t] = Y[(t / n) * ld + t % n];
    if (!do_g) return;   // (mixed form) G is formed on the tensor cores by k_g_umma
    // G[s][c] = sum_x C[virt[s]][x] AinvT[c][x]: 4 x 4 register tiles (slots x columns)
    const int ts = (nv + 3) / 4, tc = (n + 3) / 4;
    for (int tile = tid; tile < ts * tc; tile += nt) {
        const int s0 = (tile / tc) * 4, c0 = (tile % tc) * 4;
        real acc[4][4] = {};
        const real *cr[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) cr[i] = C + (size_t)s_virt[min(s0 + i, nv - 1)] * n;
        for (int x = 0; x < n; ++x) {
            real a[4], bb[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = __ldg(cr[i] + x);
#pragma unroll
            for (int j = 0; j < 4; ++j) bb[j] = Y[min(c0 + j, n - 1) * ld + x];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (s0 + i < nv && c0 + j < n) G[gofs + (size_t)(s0 + i) * n + c0 + j] = acc[i][j];
    }
}

template <typename real, int R>
cudaError_t launch_gj_r(vmc_ctx *ctx, const vmc_walkers *Wk, const real *Ca, const real *Cb, int do_g) {
    const int na = Wk->n_alpha, nb = Wk->n_beta, nmax = na > nb ? na : nb;
    const size_t smem = sizeof(real) * (size_t)nmax * (nmax + 1) + 16;
    cudaError_t e = cudaFuncSetAttribute(k_refresh_gj<real, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_refresh_gj<real, R><<<dim3(Wk->W, 2), kGJ * kGJ, smem, ctx->stream>>>(
        Wk->M, na, nb, Ca, Cb, Wk->occ_list, Wk->virt_list, Wk->pos, Wk->occ_bits, (real *)Wk->G,
        (real *)Wk->AinvT, ctx->d_status, do_g);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_gj(vmc_ctx *ctx, const vmc_walkers *Wk, const real *Ca, const real *Cb, int do_g) {
    const int nmax = Wk->n_alpha > Wk->n_beta ? Wk->n_alpha : Wk->n_beta;
    const int R = (nmax + kGJ - 1) / kGJ;
    if (R <= 2) return launch_gj_r<real, 2>(ctx, Wk, Ca, Cb, do_g);
    if (R <= 4) return launch_gj_r<real, 4>(ctx, Wk, Ca, Cb, do_g);
    if (R == 5) return launch_gj_r<real, 5>(ctx, Wk, Ca, Cb, do_g);
    if (R == 6) return launch_gj_r<real, 6>(ctx, Wk, Ca, Cb, do_g);
    return launch_gj_r<real, 8>(ctx, Wk, Ca, Cb, do_g);
}

__global__ void k_convert_c(int M, int na, int nb, const double *__restrict__ Ca, const double *__restrict__ Cb,
                            float *__restrict__ Cf) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int nA = M * na;
    if (t < nA) Cf[t] = (float)Ca[t];
    else if (t < nA + M * nb) Cf[t] = (float)Cb[t - nA];
}

// Jastrow sums S_p, and (full init only) Fock sums and the diagonal energy.
// Jastrow sums S_p = sum_{k occ, k != p} J_kp for a block of kSumWalkers walkers (thread = p): each
// walker's occupied rows of the symmetric J copy are added in ascending order, one add per
// occupied orbital (the rows are L2 resident).
// (Full init only:) Fock sums F and the diagonal energy, one walker per block.
constexpr int kSumWalkers = 8;

template <typename real>
__global__ void __launch_bounds__(VMC_THREADS)
k_jastrow_sums(int W, int M, const real *__restrict__ Jsym, const uint32_t *__restrict__ occ_bits, real *S) {
    const int N2 = 2 * M, nw = (M + 31) / 32, w0 = blockIdx.x * kSumWalkers;
    __shared__ uint32_t bits[kSumWalkers][2 * (VMC_MAX_M / 32)];
    for (int t = threadIdx.x; t < kSumWalkers * 2 * nw; t += blockDim.x) {
        const int k = t / (2 * nw), q = t % (2 * nw);
        bits[k][q] = (w0 + k < W) ? occ_bits[(size_t)(w0 + k) * 2 * nw + q] : 0u;
    }
    __syncthreads();
    for (int p = threadIdx.x; p < N2; p += blockDim.x) {
        const real jd = Jsym[(size_t)p * N2 + p];
        const int sp = p >= M, kp = p - sp * M;
        for (int k = 0; k < kSumWalkers; ++k) {
            if (w0 + k >= W) break;
            // only the walker's occupied spin orbitals r, in ascending order (the set bits of its
            // alpha words, then of its beta words): one add each, four row loads in flight at a time
            real acc = 0;
            for (int q = 0; q < 2 * nw; ++q) {
                uint32_t word = bits[k][q];
                const int base = q < nw ? 32 * q : M + 32 * (q - nw);
                while (word) {
                    int r[4], m = 0;
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (word) {
                            r[u] = base + __ffs(word) - 1;
                            word &= word - 1u;
                            m = u + 1;
                        }
                    real j[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) j[u] = u < m ? Jsym[(size_t)r[u] * N2 + p] : real(0);
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (u < m) acc += j[u];
                }
            }
            const bool occp = (bits[k][sp * nw + (kp >> 5)] >> (kp & 31)) & 1u;
            S[(size_t)(w0 + k) * N2 + p] = occp ? acc - jd : acc;
        }
    }
}

template <typename real>
__global__ void __launch_bounds__(VMC_THREADS)
k_init_sums(ListsView L, int na, int nb, const real *__restrict__ Jsym, const uint16_t *occ_list,
            real *S, double *F, double *e_diag, int full, int do_f) {
    const int w = blockIdx.x, M = L.M, ne = na + nb;
    const int tid = threadIdx.x, nt = blockDim.x;
    __shared__ int s_so[2 * VMC_MAX_M];   // occupied spin orbitals
    __shared__ double red[VMC_WARPS];
    const uint16_t *occ = occ_list + (size_t)w * ne;
    for (int c = tid; c < ne; c += nt) s_so[c] = (c < na ? 0 : M) + occ[c];
    __syncthreads();
    (void)Jsym; (void)S;
    if (!full) return;
    // F[s][e] = h_ai + sum_{j occ, spin s} Tjk[j][e] + sum_{j occ, other spin} Tj[j][e]  (FP64 form)
    for (int64_t e = tid; do_f && e < L.ns_pad; e += nt) {
        if (e >= L.ns) {
            F[((size_t)w * 2) * L.ns_pad + e] = 0.0;
            F[((size_t)w * 2 + 1) * L.ns_pad + e] = 0.0;
            continue;
        }
        const int i = (int)L.s_owner[e], a = L.s_a[e];
        const double h = L.h1[(size_t)a * M + i];
        for (int s = 0; s < 2; ++s) {
            double acc = h;
            for (int c = 0; c < ne; ++c) {
                const int js = c < na ? 0 : 1;
                const int j = occ[c];
                acc += (js == s ? L.Tjk : L.Tj)[(size_t)j * L.ns_pad + e];
            }
            F[((size_t)w * 2 + s) * L.ns_pad + e] = acc;
        }
    }
    // e_diag = e_core + sum_p h_pp + 1/2 sum_{p != q} [(pp|qq) - delta_s (pq|qp)]
    double part = 0.0;
    for (int t = tid; t < ne * ne; t += nt) {
        const int x = t / ne, y = t % ne;
        const int p = s_so[x], q = s_so[y];
        const int kp = p % M, kq = q % M;
        if (x == y) {
            part += L.hd[kp];
        } else {
            double d = L.Jd[(size_t)kp * M + kq];
            if ((p >= M) == (q >= M)) d -= L.Kd[(size_t)kp * M + kq];
            part += 0.5 * d;
        }
    }
    part = warp_sum_f64(part);
    if ((tid & 31) == 0) red[tid >> 5] = part;
    __syncthreads();
    if (tid == 0) {
        double s = L.e_core;
        for (int k = 0; k < (nt >> 5); ++k) s += red[k];
        e_diag[w] = s;
    }
}

__global__ void __launch_bounds__(VMC_THREADS)
k_log_psi(int M, int na, int nb, const double *__restrict__ Ca, const double *__restrict__ Cb,
          const double *__restrict__ J, const uint16_t *occ_list, double *out, unsigned *status) {
    const int w = blockIdx.x, ne = na + nb, N2 = 2 * M;
    const int tid = threadIdx.x, nt = blockDim.x;
    extern __shared__ double sm[];
    __shared__ int s_so[2 * VMC_MAX_M];
    __shared__ int s_piv;
    __shared__ double red[VMC_WARPS];
    const uint16_t *occ = occ_list + (size_t)w * ne;
    for (int c = tid; c < ne; c += nt) s_so[c] = (c < na ? 0 : M) + occ[c];
    __syncthreads();
    // ln C[n] = sum_{p<q} J_pq n_p n_q + sum_p J_pp n_p over the occupied spin orbitals
    double part = 0.0;
    for (int t = tid; t < ne * ne; t += nt) {
        const int x = t / ne, y = t % ne;
        if (y < x) continue;
        part += jget(J, N2, s_so[x], s_so[y]);
    }
    part = warp_sum_f64(part);
    if ((tid & 31) == 0) red[tid >> 5] = part;
    __syncthreads();
    double total = 0.0;
    if (tid == 0)
        for (int k = 0; k < (nt >> 5); ++k) total += red[k];
    int sgn_total = 1;
    for (int sg = 0; sg < 2; ++sg) {
        const int n = sg ? nb : na;
        if (n == 0) continue;
        const double *C = sg ? Cb : Ca;
        const int ld = n + 1;
        __syncthreads();
        for (int t = tid; t < n * n; t += nt) {
            const int r = t / n, x = t % n;
            sm[r * ld + x] = C[(size_t)occ[(sg ? na : 0) + r] * n + x];
        }
        __syncthreads();
        double la;
        int sgn;
        lu_logdet(sm, n, ld, &s_piv, nullptr, &la, &sgn);
        if (tid == 0) {
            total += la;
            sgn_total *= sgn;
        }
    }
    if (tid == 0) {
        if (sgn_total == 0) {
            atomicOr(status, VMC_DEV_SINGULAR);
            out[w] = -INFINITY;
        } else {
            out[w] = total;
        }
    }
}

}  // namespace

vmc_status launch_init_walkers(vmc_ctx *ctx, vmc_lists *L, const vmc_params *P, vmc_walkers *Wk,
                               int full) {
    const int M = Wk->M, na = Wk->n_alpha, nb = Wk->n_beta;
    const int nmax = na > nb ? na : nb;
    const size_t smem = sizeof(double) * ((size_t)2 * nmax * (nmax + 1) + nmax + 1);
    vmc_status st = launch_refresh_jastrow(ctx, L, P->J);
    if (st) return st;
    dim3 grid(Wk->W, 2);
    cudaError_t e;
    // register Gauss-Jordan: the FP64 form, or the mixed form when FP32 elimination is asked for;
    // otherwise the shared-memory kernels (mixed: FP64 LU, FP32 inverse from the factors)
    const bool reg = !ctx->refresh_smem && (Wk->precision == VMC_FP64 || ctx->mixed_gj32);
    if (reg) {
        if (nmax > kGJ * 8) return set_err(ctx, VMC_ERR_ARG, "n_sigma too large for the register inverse (max 128)");
        if (Wk->precision == VMC_FP64) {
            const bool oz = ctx->g_tensor_cores && g_ozaki_ok(M, na, nb);
            e = launch_gj<double>(ctx, Wk, P->C_alpha, P->C_beta, oz ? 0 : 1);
            if (e == cudaSuccess && oz) {
                vmc_status st2 = launch_g_ozaki(ctx, Wk, P->C_alpha, P->C_beta, L->cdig);
                if (st2) return st2;
            }
        } else {
            float *Cf = (float *)L->cf;
            k_convert_c<<<(M * (na + nb) + 255) / 256, 256, 0, ctx->stream>>>(M, na, nb, P->C_alpha, P->C_beta, Cf);
            ctx->launches += 1;
            const bool umma = ctx->g_tensor_cores && g_umma_smem(M, na, nb) > 0;
            e = launch_gj<float>(ctx, Wk, Cf, Cf + (size_t)M * na, umma ? 0 : 1);
            if (e == cudaSuccess && umma) {
                vmc_status st2 = launch_g_umma(ctx, Wk, Cf);
                if (st2) return st2;
            }
        }
    } else if (Wk->precision == VMC_FP64 && smem > 227 * 1024) {
        return set_err(ctx, VMC_ERR_ARG, "n_sigma too large for the in-SM inverse (max 118)");
    } else if (Wk->precision == VMC_MIXED && nmax > VMC_MAX_M / 2) {   // per-thread staging array bound
        return set_err(ctx, VMC_ERR_ARG, "n_sigma too large for the in-SM FP64 LU (max 128)");
    } else if (Wk->precision == VMC_FP64) {
        e = cudaFuncSetAttribute(k_init_tables<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            k_init_tables<double><<<grid, VMC_THREADS, smem, ctx->stream>>>(
                M, na, nb, P->C_alpha, P->C_beta, Wk->occ_list, Wk->virt_list, Wk->pos, Wk->occ_bits,
                (double *)Wk->G, (double *)Wk->AinvT, ctx->d_status);
    } else {
        const size_t smem_m = sizeof(double) * (size_t)nmax * (nmax + 1) + 16;
        float *Cf = (float *)L->cf;
        k_convert_c<<<(M * (na + nb) + 255) / 256, 256, 0, ctx->stream>>>(M, na, nb, P->C_alpha, P->C_beta, Cf);
        ctx->launches += 1;
        const bool umma = ctx->g_tensor_cores && g_umma_smem(M, na, nb) > 0;
        e = cudaFuncSetAttribute(k_init_tables_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_m);
        if (e == cudaSuccess)
            k_init_tables_mixed<<<grid, VMC_THREADS, smem_m, ctx->stream>>>(
                M, na, nb, P->C_alpha, P->C_beta, Cf, Wk->occ_list, Wk->virt_list, Wk->pos, Wk->occ_bits,
                (float *)Wk->G, (float *)Wk->AinvT, ctx->d_status, umma ? 0 : 1);
        if (e == cudaSuccess && umma) {
            vmc_status st2 = launch_g_umma(ctx, Wk, Cf);
            if (st2) return st2;
        }
    }
    ctx->launches += 1;
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(ctx, e, "k_init_tables");
    const double *js64 = (const double *)L->jsym;
    const float *js32 = (const float *)(js64 + 4 * (size_t)M * M);
    const int sb = (Wk->W + kSumWalkers - 1) / kSumWalkers;
    if (Wk->precision == VMC_FP64)
        k_jastrow_sums<double><<<sb, VMC_THREADS, 0, ctx->stream>>>(Wk->W, M, js64, Wk->occ_bits, (double *)Wk->S);
    else
        k_jastrow_sums<float><<<sb, VMC_THREADS, 0, ctx->stream>>>(Wk->W, M, js32, Wk->occ_bits, (float *)Wk->S);
    ctx->launches += 1;
    if (Wk->precision == VMC_MIXED && L->view.ns_pad > 0) {
        dim3 fg((unsigned)((L->view.ns_pad + kFockThreads - 1) / kFockThreads),
                (unsigned)((Wk->W + kFockWalkers - 1) / kFockWalkers));
        k_fock_sums_f32<<<fg, kFockThreads, 0, ctx->stream>>>(L->view, Wk->W, Wk->occ_bits, (float *)Wk->F);
        ctx->launches += 1;
    }
    if (full) {
        k_init_sums<double><<<Wk->W, VMC_THREADS, 0, ctx->stream>>>(
            L->view, na, nb, js64, Wk->occ_list, nullptr, (double *)Wk->F, Wk->e_diag, 1,
            Wk->precision == VMC_FP64 ? 1 : 0);
        ctx->launches += 1;
    }
    return cuda_check(ctx, cudaGetLastError(), "k_jastrow_sums/k_init_sums");
}

vmc_status launch_log_psi(vmc_ctx *ctx, const vmc_walkers *Wk, const vmc_params *P, double *out) {
    const int nmax = Wk->n_alpha > Wk->n_beta ? Wk->n_alpha : Wk->n_beta;
    const size_t smem = sizeof(double) * ((size_t)nmax * (nmax + 1) + 1);
    cudaError_t e = cudaFuncSetAttribute(k_log_psi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        k_log_psi<<<Wk->W, VMC_THREADS, smem, ctx->stream>>>(Wk->M, Wk->n_alpha, Wk->n_beta, P->C_alpha,
                                                             P->C_beta, P->J, Wk->occ_list, out,
                                                             ctx->d_status);
    ctx->launches += 1;
    if (e == cudaSuccess) e = cudaGetLastError();
    return cuda_check(ctx, e, "k_log_psi");
}
