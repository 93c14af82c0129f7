/*
 * Oracle for the screened orbital-space VMC hot path -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, FP64 CPU code that states what the GPU path must compute.  Only the tests,
 * the package's smoke() check and the CPU-baseline leg of the benchmark may call it; the
 * product path never does.  It shares no code with the CUDA library.
 *
 * Paper: Sabzevari & Sharma, "Improved speed and scaling in orbital space variational
 * Monte Carlo" (arXiv:1807.10633).
 *
 *   local energy        E_L[n, eps] = sum_m^eps H_nm psi(m)/psi(n)         Sec. II.A, Eq. (eloc:hci)
 *   doubles screen      keep ij->ab iff |<ab|ij> - <ab|ji>| > eps            Sec. II.A
 *   singles screen      keep i->a  iff S_ia = |<i|a>| + sum_j |<ij|aj>-<ij|ja>| > eps   Sec. II.A
 *   wavefunction        psi(n) = C[n] det(theta[n]); C = pair Jastrow        Sec. III.A
 *   CTMC                r(m<-n) = |psi(m)/psi(n)|, t_n = 1/sum r, pick m ~ r  Sec. II.B, Eq. (rate)
 *   gradient ratios     d ln psi / d p                                        Sec. III.B
 *   AMSGrad             Eqs. (m1), (m2)                                       Sec. II.C
 *
 * Everything here is done the direct way:
 *   - excitations are enumerated from the integral tensor itself (never from sorted lists);
 *   - H_nm carries the canonical fermionic phase obtained by applying annihilation and
 *     creation operators to the occupation-number vector;
 *   - psi(m)/psi(n) is a ratio of canonically ordered determinants, taken either from a
 *     table G = theta * theta[n]^-1 recomputed by LU for every call (times the row
 *     permutation sign) or, in "direct" mode, from two LU determinants;
 *   - the Jastrow ratio is exp(lnC[m] - lnC[n]) with both sums evaluated in full.
 *
 * Readings where the paper is silent (each also listed in the project design notes):
 *   - pair Jastrow lnC[n] = sum_{p<q} J_pq n_p n_q + sum_p J_pp n_p over spin orbitals,
 *     J read from its upper triangle (p <= q);
 *   - the sum over j in S_ia runs over all spin orbitals; thresholds are strict (> eps);
 *   - canonical move order: singles by (i ascending, S_ia descending, a ascending), then
 *     doubles by ((i,j) lexicographic, |<ab||ij>| descending, (a,b) ascending);
 *   - CTMC choice: q_k = floor(r_k * 2^64) as an exact 128-bit integer, Q = sum q_k,
 *     U = first word of Philox4x64-10(key = (seed, walker), counter = (step, 0, 0, 0)),
 *     T = floor(U * Q / 2^64); the first move with prefix sum > T is taken;
 *     t_n = 1 / (double(Q_hi) + double(Q_lo) * 2^-64);
 *   - AMSGrad as printed (beta1 weights the new gradient), no bias correction, dp = 0
 *     where n = 0.
 *
 * Spin-orbital index p = sigma*M + k (alpha block first).  Integrals are chemists' (pq|rs)
 * over real orbitals; the physicists' <pq|rs> of the paper equals (pr|qs) when the spins
 * match and 0 otherwise.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

typedef struct {
    int M, n_alpha, n_beta;
    const double *h1;   /* M*M */
    const double *eri;  /* M^4, (pq|rs) at ((p*M+q)*M+r)*M+s */
    double e_core;
    const double *J;    /* (2M)*(2M), read for p <= q */
    const double *Ca;   /* M*n_alpha */
    const double *Cb;   /* M*n_beta */
    /* Correlator product (Sec. III.A), optional (n_corr = 0: none).  Correlator l covers the
       spatial sites corr_sites[corr_off[l] .. corr_off[l+1]) and holds 4^k coefficients at
       corr_val[val_off[l] ..], indexed by sum_t (n_alpha(site_t) + 2 n_beta(site_t)) 4^t. */
    int n_corr;
    const int *corr_off;      /* n_corr + 1 */
    const int *corr_sites;
    const long *val_off;      /* n_corr + 1 */
    const double *corr_val;
} orc_system;

typedef struct {
    int32_t kind;       /* 1 single, 2 double */
    int32_t i, j, a, b; /* spin orbitals; j = b = -1 for singles */
    double h;           /* <m|H|n> with canonical phase */
    double ratio;       /* psi(m)/psi(n) for canonical m */
    double key;         /* screening magnitude (S_ia or |<ab||ij>|) */
} orc_move;

/* ---------------------------------------------------------------- integrals in spin orbitals */
static inline double chem(const orc_system *s, int p, int q, int r, int t) {
    const size_t M = (size_t)s->M;
    return s->eri[((p * M + q) * M + r) * M + t];
}
static inline int spin_of(const orc_system *s, int p) { return p >= s->M; }
static inline int spat(const orc_system *s, int p) { return p % s->M; }

/* physicists' <pq|rs> over spin orbitals = (pr|qs) delta(s_p,s_r) delta(s_q,s_s) */
static double phys(const orc_system *s, int p, int q, int r, int t) {
    if (spin_of(s, p) != spin_of(s, r) || spin_of(s, q) != spin_of(s, t)) return 0.0;
    return chem(s, spat(s, p), spat(s, r), spat(s, q), spat(s, t));
}
static double phys_anti(const orc_system *s, int p, int q, int r, int t) {
    return phys(s, p, q, r, t) - phys(s, p, q, t, r);
}
static double h1so(const orc_system *s, int p, int q) {
    if (spin_of(s, p) != spin_of(s, q)) return 0.0;
    return s->h1[(size_t)spat(s, p) * s->M + spat(s, q)];
}

/* ---------------------------------------------------------------- fermionic operators */
/* a_p |n>: returns the phase (+1/-1) and clears n_p, or 0 if n_p == 0 */
static int op_ann(uint8_t *n, int p) {
    if (!n[p]) return 0;
    int c = 0;
    for (int k = 0; k < p; ++k) c += n[k];
    n[p] = 0;
    return (c & 1) ? -1 : 1;
}
/* a_p^dagger |n>: returns the phase and sets n_p, or 0 if n_p == 1 */
static int op_cre(uint8_t *n, int p) {
    if (n[p]) return 0;
    int c = 0;
    for (int k = 0; k < p; ++k) c += n[k];
    n[p] = 1;
    return (c & 1) ? -1 : 1;
}

/* ---------------------------------------------------------------- dense linear algebra */
/* LU with partial pivoting of an n x n row-major matrix, in place.  Returns the sign of the
   row permutation (0 if a zero pivot was met); piv[k] = row swapped into position k. */
static int lu_factor(double *A, int n, int *piv) {
    int sgn = 1;
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = fabs(A[(size_t)k * n + k]);
        for (int r = k + 1; r < n; ++r) {
            double v = fabs(A[(size_t)r * n + k]);
            if (v > best) { best = v; p = r; }
        }
        piv[k] = p;
        if (best == 0.0) return 0;
        if (p != k) {
            for (int c = 0; c < n; ++c) {
                double t = A[(size_t)k * n + c];
                A[(size_t)k * n + c] = A[(size_t)p * n + c];
                A[(size_t)p * n + c] = t;
            }
            sgn = -sgn;
        }
        double d = A[(size_t)k * n + k];
        for (int r = k + 1; r < n; ++r) {
            double f = A[(size_t)r * n + k] / d;
            A[(size_t)r * n + k] = f;
            for (int c = k + 1; c < n; ++c) A[(size_t)r * n + c] -= f * A[(size_t)k * n + c];
        }
    }
    return sgn;
}

static double det_of(const double *A_in, int n, double *work, int *piv) {
    if (n == 0) return 1.0;
    memcpy(work, A_in, sizeof(double) * (size_t)n * n);
    int sgn = lu_factor(work, n, piv);
    if (sgn == 0) return 0.0;
    double d = (double)sgn;
    for (int k = 0; k < n; ++k) d *= work[(size_t)k * n + k];
    return d;
}

/* inverse of an n x n matrix from its LU factors (solves A X = I column by column) */
static int invert(const double *A_in, int n, double *Ainv, double *work, int *piv) {
    memcpy(work, A_in, sizeof(double) * (size_t)n * n);
    if (lu_factor(work, n, piv) == 0) return -1;
    for (int col = 0; col < n; ++col) {
        double *x = Ainv; /* column col of the inverse, stored row-major */
        double *b = (double *)malloc(sizeof(double) * n);
        for (int r = 0; r < n; ++r) b[r] = (r == col) ? 1.0 : 0.0;
        for (int k = 0; k < n; ++k) { /* apply the row swaps in order */
            int p = piv[k];
            if (p != k) { double t = b[k]; b[k] = b[p]; b[p] = t; }
        }
        for (int r = 0; r < n; ++r) /* forward: L has a unit diagonal */
            for (int c = 0; c < r; ++c) b[r] -= work[(size_t)r * n + c] * b[c];
        for (int r = n - 1; r >= 0; --r) { /* backward: U */
            for (int c = r + 1; c < n; ++c) b[r] -= work[(size_t)r * n + c] * b[c];
            b[r] /= work[(size_t)r * n + r];
        }
        for (int r = 0; r < n; ++r) x[(size_t)r * n + col] = b[r];
        free(b);
    }
    return 0;
}

/* ---------------------------------------------------------------- wavefunction */
static double jastrow_log(const orc_system *s, const uint8_t *n) {
    const int N2 = 2 * s->M;
    double acc = 0.0;
    for (int p = 0; p < N2; ++p) {
        if (!n[p]) continue;
        acc += s->J[(size_t)p * N2 + p];
        for (int q = p + 1; q < N2; ++q)
            if (n[q]) acc += s->J[(size_t)p * N2 + q];
    }
    return acc;
}

/* Fock-state index of correlator l in determinant n: site t contributes n_alpha + 2 n_beta
   times 4^t */
static long corr_index(const orc_system *s, const uint8_t *n, int l) {
    long idx = 0, w = 1;
    for (int e = s->corr_off[l]; e < s->corr_off[l + 1]; ++e, w *= 4) {
        const int site = s->corr_sites[e];
        idx += w * (n[site] + 2 * n[s->M + site]);
    }
    return idx;
}

/* C[n] = product over the correlators of c_l[n_l]  (1 without correlators) */
static double cps_value(const orc_system *s, const uint8_t *n) {
    double v = 1.0;
    for (int l = 0; l < s->n_corr; ++l) v *= s->corr_val[s->val_off[l] + corr_index(s, n, l)];
    return v;
}

/* occupied spatial orbitals of spin sigma in ascending order */
static int occ_of_spin(const orc_system *s, const uint8_t *n, int sigma, int *occ) {
    int c = 0;
    for (int k = 0; k < s->M; ++k)
        if (n[sigma * s->M + k]) occ[c++] = k;
    return c;
}

static double slater_det(const orc_system *s, const uint8_t *n, int sigma, double *work, double *work2, int *piv) {
    const int ns = sigma ? s->n_beta : s->n_alpha;
    const double *C = sigma ? s->Cb : s->Ca;
    int *occ = (int *)malloc(sizeof(int) * (s->M + 1));
    int c = occ_of_spin(s, n, sigma, occ);
    double d = 0.0;
    if (c == ns) {
        for (int r = 0; r < ns; ++r)
            for (int x = 0; x < ns; ++x) work[(size_t)r * ns + x] = C[(size_t)occ[r] * ns + x];
        d = det_of(work, ns, work2, piv);
    }
    free(occ);
    return d;
}

/* psi(n) = exp(lnJ[n]) C[n] det C^alpha[n] det C^beta[n]  (Sec. III.A: the pair Jastrow and, when
   present, the correlator product) */
double orc_psi(const orc_system *s, const uint8_t *n) {
    const int nmax = (s->n_alpha > s->n_beta ? s->n_alpha : s->n_beta) + 1;
    double *w1 = (double *)malloc(sizeof(double) * nmax * nmax);
    double *w2 = (double *)malloc(sizeof(double) * nmax * nmax);
    int *piv = (int *)malloc(sizeof(int) * nmax);
    double da = slater_det(s, n, 0, w1, w2, piv);
    double db = slater_det(s, n, 1, w1, w2, piv);
    double r = exp(jastrow_log(s, n)) * da * db;
    if (s->n_corr) r *= cps_value(s, n);
    free(w1); free(w2); free(piv);
    return r;
}

/* Per-spin tables for one determinant: canonical occupied list, G = C * C_occ^-1 (M x ns),
   and C_occ^-1 (ns x ns).  Returns 0, or -1 if C_occ is singular. */
typedef struct {
    int ns[2];
    int occ[2][512];
    int pos[2][512];      /* canonical row position of an occupied spatial orbital, else -1 */
    double *G[2];         /* M x ns */
    double *Ainv[2];      /* ns x ns: Ainv[x][c] */
} det_tables;

static int tables_build(const orc_system *s, const uint8_t *n, det_tables *t) {
    for (int sg = 0; sg < 2; ++sg) {
        const int ns = sg ? s->n_beta : s->n_alpha;
        const double *C = sg ? s->Cb : s->Ca;
        t->ns[sg] = ns;
        t->G[sg] = (double *)calloc((size_t)s->M * ns + 1, sizeof(double));
        t->Ainv[sg] = (double *)calloc((size_t)ns * ns + 1, sizeof(double));
        int c = occ_of_spin(s, n, sg, t->occ[sg]);
        if (c != ns) return -1;
        for (int k = 0; k < s->M; ++k) t->pos[sg][k] = -1;
        for (int r = 0; r < ns; ++r) t->pos[sg][t->occ[sg][r]] = r;
        if (ns <= 0) continue;
        const size_t nn = (size_t)ns;
        double *A = (double *)malloc(sizeof(double) * nn * nn);
        double *work = (double *)malloc(sizeof(double) * nn * nn);
        int *piv = (int *)malloc(sizeof(int) * nn);
        for (int r = 0; r < ns; ++r)
            for (int x = 0; x < ns; ++x) A[(size_t)r * ns + x] = C[(size_t)t->occ[sg][r] * ns + x];
        int rc = invert(A, ns, t->Ainv[sg], work, piv);
        free(A); free(work); free(piv);
        if (rc) return -1;
        for (int k = 0; k < s->M; ++k)
            for (int cc = 0; cc < ns; ++cc) {
                double acc = 0.0;
                for (int x = 0; x < ns; ++x) acc += C[(size_t)k * ns + x] * t->Ainv[sg][(size_t)x * ns + cc];
                t->G[sg][(size_t)k * ns + cc] = acc;
            }
    }
    return 0;
}
static void tables_free(det_tables *t) {
    for (int sg = 0; sg < 2; ++sg) { free(t->G[sg]); free(t->Ainv[sg]); }
}

/* Canonical-order determinant ratio det theta[m] / det theta[n] within one spin, for m obtained
   by replacing the occupied orbitals from[0..k) by to[0..k) (k = 1 or 2, sorted rows in m).
   Computed as the in-place replacement ratio (a minor of G, Eq. (R)) times the sign of the
   permutation that sorts the replaced rows. */
static double spin_ratio(const det_tables *t, int sg, int k, const int *from, const int *to, int M) {
    const int ns = t->ns[sg];
    const double *G = t->G[sg];
    /* rows of the in-place matrix: occupied list with from[] replaced by to[] */
    int *rows = (int *)malloc(sizeof(int) * (ns + 1));
    for (int r = 0; r < ns; ++r) rows[r] = t->occ[sg][r];
    int cols[2];
    for (int e = 0; e < k; ++e) {
        cols[e] = t->pos[sg][from[e]];
        rows[cols[e]] = to[e];
    }
    double minor;
    if (k == 1) minor = G[(size_t)to[0] * ns + cols[0]];
    else minor = G[(size_t)to[0] * ns + cols[0]] * G[(size_t)to[1] * ns + cols[1]]
               - G[(size_t)to[0] * ns + cols[1]] * G[(size_t)to[1] * ns + cols[0]];
    /* parity of sorting rows[] (count inversions) */
    int inv = 0;
    for (int x = 0; x < ns; ++x)
        for (int y = x + 1; y < ns; ++y)
            if (rows[x] > rows[y]) ++inv;
    free(rows);
    (void)M;
    return (inv & 1) ? -minor : minor;
}

/* ---------------------------------------------------------------- screening quantities */
/* S_ia = |<i|h|a>| + sum_{j in all spin orbitals} |<ij|aj> - <ij|ja>|   (Sec. II.A).
   The sum visits the spin orbitals of i's spin first, then the other spin (each ascending), so
   that an alpha and a beta single with the same spatial orbitals get bit-identical bounds. */
static double singles_bound(const orc_system *s, int i, int a) {
    double acc = fabs(h1so(s, i, a));
    const int M = s->M, si = spin_of(s, i);
    for (int t = 0; t < 2; ++t) {
        const int sj = t == 0 ? si : 1 - si;
        for (int k = 0; k < M; ++k) {
            const int j = sj * M + k;
            acc += fabs(phys(s, i, j, a, j) - phys(s, i, j, j, a));
        }
    }
    return acc;
}

/* ---------------------------------------------------------------- move ordering */
static int move_cmp(const void *pa, const void *pb) {
    const orc_move *x = (const orc_move *)pa, *y = (const orc_move *)pb;
    if (x->kind != y->kind) return x->kind - y->kind;           /* singles first */
    if (x->i != y->i) return x->i - y->i;
    if (x->kind == 2 && x->j != y->j) return x->j - y->j;
    if (x->key != y->key) return x->key > y->key ? -1 : 1;      /* magnitude descending */
    if (x->a != y->a) return x->a - y->a;
    return x->b - y->b;
}

/* ---------------------------------------------------------------- local energy */
/*
 * E_L[n, eps] of Eq. (eloc:hci) for the determinant with occupation numbers n[0..2M).
 * Writes the screened connected determinants, in canonical order, to moves[0..cap) (when
 * moves != NULL) and returns their number; returns -1 if C_occ is singular, -2 on overflow.
 * direct != 0 takes every psi(m)/psi(n) as a ratio of two determinants instead of from G.
 */
long orc_local_energy(const orc_system *s, const uint8_t *n_in, double eps, int direct,
                      double *e_loc, double *e_diag_out, orc_move *moves, long cap) {
    const int M = s->M, N2 = 2 * M;
    uint8_t *n = (uint8_t *)malloc(N2);
    uint8_t *m = (uint8_t *)malloc(N2);
    memcpy(n, n_in, N2);

    det_tables t;
    memset(&t, 0, sizeof(t));
    if (tables_build(s, n, &t)) { tables_free(&t); free(n); free(m); return -1; }
    const double lnC_n = jastrow_log(s, n);
    const double cps_n = cps_value(s, n);
    const double psi_n = direct ? orc_psi(s, n) : 0.0;

    /* diagonal: E_core + sum_i h_ii + 1/2 sum_{i != j} <ij||ij> */
    double ed = s->e_core;
    for (int i = 0; i < N2; ++i) {
        if (!n[i]) continue;
        ed += h1so(s, i, i);
        for (int j = 0; j < N2; ++j)
            if (n[j] && j != i) ed += 0.5 * phys_anti(s, i, j, i, j);
    }

    long nm = 0;
    int overflow = 0;
    double acc = 0.0;

    /* singles i -> a, same spin, S_ia > eps */
    for (int i = 0; i < N2; ++i) {
        if (!n[i]) continue;
        for (int a = 0; a < N2; ++a) {
            if (n[a] || spin_of(s, a) != spin_of(s, i)) continue;
            double key = singles_bound(s, i, a);
            if (!(key > eps)) continue;
            memcpy(m, n, N2);
            int ph = op_ann(m, i);
            ph *= op_cre(m, a);
            double hel = h1so(s, a, i);
            for (int j = 0; j < N2; ++j)
                if (n[j]) hel += phys_anti(s, a, j, i, j);
            hel *= ph;
            double ratio;
            if (direct) {
                ratio = orc_psi(s, m) / psi_n;
            } else {
                int sg = spin_of(s, i);
                int from = spat(s, i), to = spat(s, a);
                ratio = spin_ratio(&t, sg, 1, &from, &to, M) * exp(jastrow_log(s, m) - lnC_n);
                if (s->n_corr) ratio *= cps_value(s, m) / cps_n;
            }
            acc += hel * ratio;
            if (moves) {
                if (nm < cap) {
                    orc_move mv = {1, i, -1, a, -1, hel, ratio, key};
                    moves[nm] = mv;
                } else overflow = 1;
            }
            ++nm;
        }
    }

    /* doubles ij -> ab, i < j occupied, a < b empty, spin conserving, |<ab||ij>| > eps */
    for (int i = 0; i < N2; ++i) {
        if (!n[i]) continue;
        for (int j = i + 1; j < N2; ++j) {
            if (!n[j]) continue;
            for (int a = 0; a < N2; ++a) {
                if (n[a]) continue;
                for (int b = a + 1; b < N2; ++b) {
                    if (n[b]) continue;
                    /* spin conservation: the multiset of spins must match */
                    if (spin_of(s, a) + spin_of(s, b) != spin_of(s, i) + spin_of(s, j)) continue;
                    double v = phys_anti(s, a, b, i, j);
                    double key = fabs(v);
                    if (!(key > eps)) continue;
                    memcpy(m, n, N2);
                    int ph = op_ann(m, i);
                    ph *= op_ann(m, j);
                    ph *= op_cre(m, b);
                    ph *= op_cre(m, a);
                    /* |m> = a+_a a+_b a_j a_i |n> up to ph; H_nm = ph <ab||ij> */
                    double hel = ph * v;
                    double ratio;
                    if (direct) {
                        ratio = orc_psi(s, m) / psi_n;
                    } else {
                        double jr = exp(jastrow_log(s, m) - lnC_n);
                        int si = spin_of(s, i), sj = spin_of(s, j);
                        if (si == sj) {
                            /* rows of the sorted m: a and b replace i and j (either pairing
                               gives the same sorted determinant) */
                            int from[2] = {spat(s, i), spat(s, j)}, to[2] = {spat(s, a), spat(s, b)};
                            ratio = spin_ratio(&t, si, 2, from, to, M) * jr;
                        } else {
                            int fa = spat(s, i), ta = spat(s, a);  /* alpha: i -> a */
                            int fb = spat(s, j), tb = spat(s, b);  /* beta:  j -> b */
                            ratio = spin_ratio(&t, 0, 1, &fa, &ta, M) *
                                    spin_ratio(&t, 1, 1, &fb, &tb, M) * jr;
                        }
                        if (s->n_corr) ratio *= cps_value(s, m) / cps_n;
                    }
                    acc += hel * ratio;
                    if (moves) {
                        if (nm < cap) {
                            orc_move mv = {2, i, j, a, b, hel, ratio, key};
                            moves[nm] = mv;
                        } else overflow = 1;
                    }
                    ++nm;
                }
            }
        }
    }
    if (moves && !overflow) qsort(moves, (size_t)nm, sizeof(orc_move), move_cmp);
    if (e_loc) *e_loc = ed + acc;
    if (e_diag_out) *e_diag_out = ed;
    tables_free(&t);
    free(n); free(m);
    return overflow ? -2 : nm;
}

/* ---------------------------------------------------------------- Philox4x64-10 */
/* Counter-based generator of Salmon, Moraes, Dror & Shaw (SC'11): ten rounds of two 64x64->128
   multiplications with the round keys bumped by the Weyl constants between rounds. */
void orc_philox4x64(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4]) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        u128 p0 = (u128)M0 * x0, p1 = (u128)M1 * x2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        uint64_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += W0; k1 += W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* ---------------------------------------------------------------- CTMC (Sec. II.B) */
/* floor(r * 2^64) as an exact 128-bit integer; r >= 0 finite and below 2^43 */
static u128 rate_fixed(double r) {
    if (!(r > 0.0)) return 0;
    int e;
    double f = frexp(r, &e);             /* r = f * 2^e, f in [0.5, 1) */
    uint64_t mant = (uint64_t)ldexp(f, 53); /* exact 53-bit integer: r = mant * 2^(e-53) */
    int sh = e - 53 + 64;                /* r * 2^64 = mant * 2^sh */
    if (sh >= 0) return ((u128)mant) << sh;
    if (sh <= -64) return 0;
    return (u128)(mant >> (-sh));
}

/*
 * Rejection-free choice among the screened moves (canonical order) with rates r_k = |ratio_k|
 * (Eq. rate).  Writes the chosen index and the residence time t_n = 1 / sum r (computed from the
 * exact integer sum).  Returns 0, 1 if no move has a non-zero fixed-point rate, 2 if a rate is
 * too large for the fixed-point range.
 */
int orc_ctmc_choose_u(const orc_move *moves, long nm, uint64_t U, long *chosen, double *t_res);

int orc_ctmc_choose(const orc_move *moves, long nm, uint64_t seed, uint64_t walker, uint64_t step,
                    long *chosen, double *t_res) {
    uint64_t ctr[4] = {step, 0, 0, 0}, key[2] = {seed, walker}, x[4];
    orc_philox4x64(ctr, key, x);
    return orc_ctmc_choose_u(moves, nm, x[0], chosen, t_res);
}

/* The same choice for a given uniform 64-bit draw U (word 0 of Philox above). */
int orc_ctmc_choose_u(const orc_move *moves, long nm, uint64_t U, long *chosen, double *t_res) {
    u128 Q = 0;
    for (long k = 0; k < nm; ++k) {
        double r = fabs(moves[k].ratio);
        if (r >= 0x1p43) return 2;
        Q += rate_fixed(r);
    }
    *chosen = -1;
    if (Q == 0) { *t_res = 0.0; return 1; }
    uint64_t qh = (uint64_t)(Q >> 64), ql = (uint64_t)Q;
    *t_res = 1.0 / ((double)qh + (double)ql * 0x1p-64);
    /* T = floor(U * Q / 2^64): U*Q = U*qh*2^64 + U*ql */
    u128 T = (u128)U * qh + (u128)(((u128)U * ql) >> 64);
    u128 pre = 0;
    for (long k = 0; k < nm; ++k) {
        pre += rate_fixed(fabs(moves[k].ratio));
        if (pre > T) { *chosen = k; return 0; }
    }
    return 1; /* unreachable when T < Q */
}

void orc_apply_move(const orc_move *mv, uint8_t *n) {
    n[mv->i] = 0;
    if (mv->kind == 2) n[mv->j] = 0;
    n[mv->a] = 1;
    if (mv->kind == 2) n[mv->b] = 1;
}

/* ---------------------------------------------------------------- gradient ratios (Sec. III.B) */
/*
 * Adds weight * d ln psi(n) / d p to the gradient buffers:
 *   dJ[p][q] (p < q) += weight * n_p n_q ;  dJ[p][p] += weight * n_p      (upper triangle)
 *   dC^sigma[k][x]   += weight * (theta[n]^-1)[x][row(k)] for occupied k  (0 otherwise)
 * Returns 0 or -1 if C_occ is singular.
 */
int orc_grad_logpsi(const orc_system *s, const uint8_t *n, double weight,
                    double *dJ, double *dCa, double *dCb) {
    const int M = s->M, N2 = 2 * M;
    for (int p = 0; p < N2; ++p) {
        if (!n[p]) continue;
        dJ[(size_t)p * N2 + p] += weight;
        for (int q = p + 1; q < N2; ++q)
            if (n[q]) dJ[(size_t)p * N2 + q] += weight;
    }
    det_tables t;
    memset(&t, 0, sizeof(t));
    if (tables_build(s, n, &t)) { tables_free(&t); return -1; }
    for (int sg = 0; sg < 2; ++sg) {
        const int ns = t.ns[sg];
        double *dC = sg ? dCb : dCa;
        for (int r = 0; r < ns; ++r) {
            int k = t.occ[sg][r];
            for (int x = 0; x < ns; ++x) dC[(size_t)k * ns + x] += weight * t.Ainv[sg][(size_t)x * ns + r];
        }
    }
    tables_free(&t);
    return 0;
}

/*
 * Adds weight * d ln psi(n) / d c_l[k] = weight * delta(k, n_l) / c_l[k] to dc (laid out like
 * corr_val): psi is linear in each coefficient, and only the coefficient of the Fock state the
 * determinant puts on the correlator's sites enters psi(n) (Sec. III.A-B).
 */
void orc_grad_cps(const orc_system *s, const uint8_t *n, double weight, double *dc) {
    for (int l = 0; l < s->n_corr; ++l) {
        const long k = s->val_off[l] + corr_index(s, n, l);
        dc[k] += weight / s->corr_val[k];
    }
}

/* ---------------------------------------------------------------- AMSGrad, Eqs. (m1), (m2) */
void orc_amsgrad(double *p, const double *g, double *m, double *v, long np,
                 double alpha, double beta1, double beta2) {
    for (long k = 0; k < np; ++k) {
        m[k] = (1.0 - beta1) * m[k] + beta1 * g[k];
        double cand = (1.0 - beta2) * v[k] + beta2 * (g[k] * g[k]);
        v[k] = v[k] > cand ? v[k] : cand;
        if (v[k] > 0.0) p[k] -= alpha * m[k] / sqrt(v[k]);
    }
}

/* ---------------------------------------------------------------- batched driver */
/*
 * One CTMC step for W walkers (occupations occ[W][2M], updated in place): E_L, choice and move.
 * e_loc[w], t_res[w] and the chosen move (kind, i, j, a, b) in mv_out[w][5] are written.
 * steps[w] is the Philox counter for walker w and is incremented.  Returns the number of
 * walkers with an error (singular determinant, no move, overflow).
 */
long orc_sweep(const orc_system *s, long W, uint8_t *occ, double eps, uint64_t seed,
               uint64_t *steps, double *e_loc, double *t_res, int32_t *mv_out, long cap,
               int n_threads) {
    long n_err = 0;
    const int N2 = 2 * s->M;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : n_err) num_threads(n_threads)
    for (long w = 0; w < W; ++w) {
        orc_move *mv = (orc_move *)malloc(sizeof(orc_move) * (size_t)cap);
        uint8_t *n = occ + (size_t)w * N2;
        double el = 0.0, ed = 0.0, tr = 0.0;
        long nm = orc_local_energy(s, n, eps, 0, &el, &ed, mv, cap);
        long k = -1;
        int rc = nm < 0 ? 3 : orc_ctmc_choose(mv, nm, seed, (uint64_t)w, steps[w], &k, &tr);
        e_loc[w] = el;
        t_res[w] = tr;
        int32_t *o = mv_out + (size_t)w * 5;
        if (rc == 0 && k >= 0) {
            o[0] = mv[k].kind; o[1] = mv[k].i; o[2] = mv[k].j; o[3] = mv[k].a; o[4] = mv[k].b;
            orc_apply_move(&mv[k], n);
        } else {
            o[0] = 0; o[1] = o[2] = o[3] = o[4] = -1;
            n_err += 1;
        }
        steps[w] += 1;
        free(mv);
    }
    return n_err;
}

/* E_L for W walkers (occ[W][2M]) in parallel; returns the number of failed walkers */
long orc_local_energy_batch(const orc_system *s, long W, const uint8_t *occ, double eps,
                            double *e_loc, double *e_diag, long *n_moves, int n_threads) {
    long n_err = 0;
    const int N2 = 2 * s->M;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : n_err) num_threads(n_threads)
    for (long w = 0; w < W; ++w) {
        double el = 0.0, ed = 0.0;
        long nm = orc_local_energy(s, occ + (size_t)w * N2, eps, 0, &el, &ed, NULL, 0);
        e_loc[w] = el;
        if (e_diag) e_diag[w] = ed;
        if (n_moves) n_moves[w] = nm;
        if (nm < 0) n_err += 1;
    }
    return n_err;
}

/* ---------------------------------------------------------------- near ties of the screen (Sec. II.A) */
/*
 * Number of screening quantities within rounding of the threshold: | |x| - eps | < 1e-12 max(1, eps),
 * where the screen keeps |x| > eps.  The items are those of the screened sums over spin orbitals,
 * independent of any determinant: S_ia for every same-spin pair i != a, and |<ab||ij>| for every
 * i < j, a < b with a, b not in {i, j} and the spins of (a, b) those of (i, j).
 */
long orc_near_ties(const orc_system *s, double eps) {
    const int N2 = 2 * s->M;
    const double band = 1e-12 * (eps > 1.0 ? eps : 1.0);
    long n = 0;
    for (int i = 0; i < N2; ++i)
        for (int a = 0; a < N2; ++a) {
            if (a == i || spin_of(s, a) != spin_of(s, i)) continue;
            if (fabs(singles_bound(s, i, a) - eps) < band) ++n;
        }
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : n)
    for (int i = 0; i < N2; ++i)
        for (int j = i + 1; j < N2; ++j)
            for (int a = 0; a < N2; ++a) {
                if (a == i || a == j) continue;
                for (int b = a + 1; b < N2; ++b) {
                    if (b == i || b == j) continue;
                    if (spin_of(s, a) + spin_of(s, b) != spin_of(s, i) + spin_of(s, j)) continue;
                    if (fabs(fabs(phys_anti(s, a, b, i, j)) - eps) < band) ++n;
                }
            }
    return n;
}
