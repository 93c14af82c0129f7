/*
 * vmc.h -- C ABI of the GB300 (sm_103a) screened orbital-space VMC hot path.
 *
 * Method: Sabzevari & Sharma, "Improved speed and scaling in orbital space variational Monte
 * Carlo" (arXiv:1807.10633).  The three tasks of Sec. II -- local energy of a determinant,
 * sampling determinants from rho = |psi|^2, optimising the parameters -- map onto the calls
 * below.  Every compute step runs in the library's CUDA kernels on one GPU.
 *
 * Conventions shared by every call
 *   - M spatial orbitals, 2M spin orbitals, spin orbital p = sigma*M + k (alpha block first).
 *   - Integrals: h1[p*M+q] = <p|h|q>; eri[((p*M+q)*M+r)*M+s] = (pq|rs) in chemists' notation
 *     (real orbitals, 8-fold symmetric).  The paper's physicists' <ab|ij> equals (ai|bj).
 *   - Wavefunction (Sec. III.A with a pair Jastrow in place of the general correlators):
 *       psi(n) = exp(sum_{p<q} J_pq n_p n_q + sum_p J_pp n_p) det C^a[n^a] det C^b[n^b].
 *     J is (2M)x(2M) row-major and is read from its upper triangle (p <= q) only.
 *     C^sigma is M x n_sigma row-major.
 *   - All pointers named d_* or stored in vmc_walkers are DEVICE pointers owned by the caller;
 *     the library never frees them.  Pointers named h_* are host pointers, read during the
 *     call only.  Work is queued on the context's stream; calls return once it is queued.
 *   - Every call returns a vmc_status.  Errors found on the device (fixed-point rate overflow,
 *     a walker with no allowed move, a singular C_occ) are latched in a device status word;
 *     vmc_sync() waits for the stream and returns the latched error (then clears it).
 *   - On an error the call leaves its outputs unspecified and vmc_last_error() describes it.
 */
#ifndef VMC_H
#define VMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    VMC_OK = 0,
    VMC_ERR_ARG = 1,       /* invalid argument, size or call order */
    VMC_ERR_CUDA = 2,      /* a CUDA runtime call failed */
    VMC_ERR_OOM = 3,       /* device or host allocation failed */
    VMC_ERR_SINGULAR = 4,  /* a C_occ block is singular (|pivot| == 0) */
    VMC_ERR_TIMEOUT = 5,   /* a bounded device wait gave up */
    VMC_ERR_OVERFLOW = 6,  /* a CTMC rate reached the fixed-point limit 2^43 */
    VMC_ERR_NOMOVE = 7     /* a walker had no move with a non-zero fixed-point rate */
} vmc_status;

typedef enum {
    VMC_FP64 = 0,          /* G, A^-1, Jastrow sums and ratios in FP64 */
    VMC_MIXED = 1          /* G, A^-1, Jastrow and Fock sums, ratios in FP32; C_occ LU and the
                              walker sums (energy, gradient) in FP64 */
} vmc_precision;

typedef struct vmc_ctx vmc_ctx;       /* device, stream, workspace, status word */
typedef struct vmc_lists vmc_lists;   /* device-resident screened integral lists */

/* Create a context on CUDA device `device`; `cuda_stream` is a cudaStream_t (NULL = legacy
   default stream).  The context allocates a small status word and grows a workspace on demand. */
vmc_status vmc_create(vmc_ctx **ctx, int device, void *cuda_stream);
vmc_status vmc_destroy(vmc_ctx *ctx);
/* Replace the stream used by later calls (cudaStream_t). */
vmc_status vmc_set_stream(vmc_ctx *ctx, void *cuda_stream);
/* Text of the last error seen on this context ("" if none); valid until the next call. */
const char *vmc_last_error(const vmc_ctx *ctx);
/* Wait for the context's stream; return and clear the latched device status. */
vmc_status vmc_sync(vmc_ctx *ctx);

/*
 * Screened integral lists in "heat-bath" form (Sec. II.A).
 *   same-spin pairs p<q : entries {a<b, v = (ap|bq) - (aq|bp)}, |v| > eps, a,b not in {p,q}
 *   opposite-spin (p_alpha, q_beta) : entries {a, b, v = (ap|bq)}, |v| > eps, a != p, b != q
 *   singles i : entries {a != i, S_ia} with S_ia = |h_ia| + sum_j |<ij|aj> - <ij|ja>| > eps
 *               (j over all spin orbitals), the bound of Sec. II.A
 * Each list is sorted by magnitude descending (ties: a, then b ascending), so a walk can stop
 * at the first entry at or below a threshold.  The library also stores, per singles entry,
 * the Coulomb/exchange columns used to keep each walker's single-excitation elements
 * h_ai + sum_{j occ} <aj||ij> up to date, and the diagonal Coulomb/exchange tables.
 *   h_h1 : [M*M] host.
 *   h_eri : host, eri_packed = 0: dense [M^4] as above; eri_packed = 1: the 8-fold packed form,
 *           (pq|rs) at PQ(PQ+1)/2 + RS for PQ >= RS, with pair index pq = p(p+1)/2 + q for
 *           p >= q (M(M+1)/2 * (M(M+1)/2 + 1) / 2 doubles; 0.66 GB instead of 5.2 GB at M = 160).
 *           Both forms give identical lists when they hold the same values.
 *   e_core : constant added to every E_L.
 *   eps  : build threshold (>= 0); later calls may walk with any eps_run >= eps.
 *   M    : 1 <= M <= 256.
 * The lists are built on the host (once per eps, O(M^4 log M)) and copied to the device.
 * Free with vmc_lists_destroy.
 */
vmc_status vmc_build_screened_lists(vmc_ctx *ctx, int M, const double *h_h1, const double *h_eri,
                                    int eri_packed, double e_core, double eps, vmc_lists **out);
vmc_status vmc_lists_destroy(vmc_lists *lists);

/* Sizes of a list object: number of singles entries (the length of each walker's per-spin
   Fock-sum vector), same-spin and opposite-spin double entries. */
vmc_status vmc_lists_info(const vmc_lists *lists, int64_t *n_singles, int64_t *n_same,
                          int64_t *n_opp);

/* Work layout of the local energy for these lists: band = the largest |p - q| of a non-empty
   pair list (the pair candidates of an orbital row), n_groups = the warp groups per walker
   (singles blocks of 32 spin orbitals and orbital-row groups, in canonical move order); the CTMC
   rate store holds one 128-bit rate sum and one FP64 energy partial per group and walker. */
vmc_status vmc_lists_layout(const vmc_lists *lists, int *band, int *n_groups);

/*
 * Near ties of the screening threshold (Sec. II.A keeps |x| > eps; an item whose magnitude lies
 * within rounding of eps could be kept or dropped by a different summation order, so it is
 * reported rather than resolved).  *n_near = the number of screening quantities x with
 * | |x| - eps | < 1e-12 max(1, eps), counted over spin orbitals: S_ia of every same-spin single
 * i -> a (a != i) and |<ab||ij>| of every spin-conserving double i<j -> a<b with a, b not in
 * {i, j}, whether or not the item is kept.  eps = the build eps: the builder's own count;
 * eps above the build eps by more than the band: counted from the stored entries; otherwise
 * VMC_ERR_ARG.  Host-only (no device work).
 */
vmc_status vmc_lists_near_ties(const vmc_lists *lists, double eps, int64_t *n_near);

/*
 * The host pass of vmc_build_screened_lists alone (no context, no device): out[0..2] = the
 * numbers of singles, same-spin and opposite-spin entries, out[3] = the near-tie count of eps (as
 * vmc_lists_near_ties), out[4] = a 64-bit FNV-1a digest of every host array the device lists are
 * made from (offsets, keys, orbitals, values, Fock and diagonal tables).  Same arguments and
 * errors as vmc_build_screened_lists.
 */
vmc_status vmc_screened_lists_summary(int M, const double *h_h1, const double *h_eri, int eri_packed,
                                      double eps, int64_t out[5]);

/*
 * Walker state (Sec. III.B): one determinant per walker and the tables that make every ratio
 * O(1).  All arrays are caller-owned device buffers of W walkers, walker-major:
 *   occ_bits  uint32 [W][2][ceil(M/32)]  occupation bit strings per spin (bit k of spatial k)
 *   occ_list  uint16 [W][na+nb]     column c -> occupied spatial orbital (alpha cols, beta cols)
 *   virt_list uint16 [W][(M-na)+(M-nb)]  virtual slot -> unoccupied spatial orbital
 *   pos       uint16 [W][2M]    spin orbital -> its column if occupied, 0x8000|slot if not
 *   G         real   [W][(M-na)*na + (M-nb)*nb]  virtual rows of G^s = C^s (C^s_occ)^-1,
 *             row = virtual slot, column = occupied column (Eq. R: G_ac = det ratio of i->a)
 *   AinvT     real   [W][na*na + nb*nb]  (C^s_occ)^-1 transposed: AinvT[c][x]
 *   S         real   [W][2M]   Jastrow sums S_p = sum_{k occ, k != p} J_pk
 *   F         real   [W][2][ns_pad]  h_ai + sum_{j occ} <aj||ij> for every singles entry
 *                     (i -> a) and spin (the elements of Sec. II.A, kept up to date per move;
 *                     ns_pad = n_singles rounded up to a multiple of 4, padding entries zero;
 *                     the mixed form recomputes them at every refresh)
 *   e_diag    double [W]       <n|H|n> including e_core
 *   rng_counter uint64 [W]     Philox counter of each walker (advanced by vmc_ctmc_step)
 * real = double for VMC_FP64, float for VMC_MIXED.  The orbital order inside occ_list and
 * virt_list is an implementation detail (moves replace entries in place).
 */
typedef struct {
    int W, M, n_alpha, n_beta;
    int precision;            /* vmc_precision of G, AinvT, S, F */
    uint32_t *occ_bits;
    uint16_t *occ_list;
    uint16_t *virt_list;
    uint16_t *pos;
    void *G;
    void *AinvT;
    void *S;
    void *F;
    double *e_diag;
    uint64_t *rng_counter;
    uint16_t *cps_state;      /* [W][n_corr] coefficient index of every correlator (only with a
                                 correlator product, see vmc_cps_create; NULL otherwise) */
} vmc_walkers;

typedef struct vmc_cps vmc_cps;       /* device copy of a correlator product's structure */

/*
 * Wavefunction parameters, device pointers: J [(2M)*(2M)], C_alpha [M*na], C_beta [M*nb].
 * Optional correlator product (Sec. III.A, the general form of the Jastrow factor): cps (NULL:
 * none) and its coefficients cps_values [n_values] (FP64, the parameters; layout in
 * vmc_cps_create).  psi(n) is then multiplied by prod_l c_l[n_l].
 */
typedef struct {
    const double *J;
    const double *C_alpha;
    const double *C_beta;
    const vmc_cps *cps;
    const double *cps_values;
} vmc_params;

/*
 * Correlator product of Sec. III.A: psi(n) = prod_l c_l[n_l] x (pair Jastrow) x det C^a det C^b.
 * Correlator l covers the spatial sites h_sites[h_off[l] .. h_off[l+1]) (1 to 8 distinct sites
 * below M; at most 16 correlators may cover one site); its coefficients are c_l[k] for
 * k = sum_t (n_alpha(site_t) + 2 n_beta(site_t)) 4^t, stored at cps_values[off_l + k] with off_l the
 * sum of 4^(sites of l') over l' < l.  The library copies the structure (h_off [n_corr + 1],
 * h_sites, host) to the device and builds per-site lists of the correlators covering each site,
 * so a move's ratio multiplies c_l[new] / c_l[old] over the correlators that touch the changed
 * orbitals (Sec. III.B) and the gradient ratio is d ln psi / d c_l[k] = 1/c_l[k] for the k present.
 * The walkers' state is one 16-bit index per correlator (vmc_walkers.cps_state), set by
 * vmc_walkers_init / vmc_walkers_refresh and kept up to date by vmc_ctmc_step.  The correlator
 * product is supported by the per-system calls (not by the batched launches).
 */
vmc_status vmc_cps_create(vmc_ctx *ctx, int M, int n_corr, const int32_t *h_off, const int32_t *h_sites,
                          vmc_cps **out);
vmc_status vmc_cps_destroy(vmc_cps *cps);
/* Number of correlators and of coefficients (the length of cps_values). */
vmc_status vmc_cps_info(const vmc_cps *cps, int *n_corr, int64_t *n_values);

/* Element counts of every walker array for W walkers (for allocation by the caller):
   out[0..9] = occ_bits, occ_list, virt_list, pos, G, AinvT, S, F, e_diag, rng_counter. */
vmc_status vmc_walkers_sizes(int W, int M, int n_alpha, int n_beta, const vmc_lists *lists,
                             int64_t out[10]);

/*
 * (Re)build every walker table from occ_list (each spin block holds the walker's occupied
 * orbitals in any order) and the parameters: occ_bits, virt_list, pos, C_occ^-1 (the one O(N^3)
 * step of Sec. III.B: FP64 Gauss-Jordan with partial pivoting for VMC_FP64, FP64 LU with partial
 * pivoting and the inverse from the factors in FP32 for VMC_MIXED; see the options below),
 * G = C C_occ^-1 (on the tensor cores for VMC_MIXED), S, F, e_diag.  Also
 * refreshes the Jastrow constants stored with the lists for these parameters.  rng_counter is
 * left as is.  This is the periodic recompute (e.g. every 64 moves, and after every parameter
 * update).  Singular blocks latch VMC_ERR_SINGULAR.
 */
vmc_status vmc_walkers_init(vmc_ctx *ctx, vmc_lists *lists, const vmc_params *params,
                            vmc_walkers *walkers);

/*
 * After a parameter update: refresh the parameter-dependent tables only (Jastrow constants of
 * the lists, C_occ^-1 as in vmc_walkers_init, G, S; the mixed form also recomputes F).  e_diag
 * depends on the occupations alone and is kept.  Same errors as vmc_walkers_init.
 */
vmc_status vmc_walkers_refresh(vmc_ctx *ctx, vmc_lists *lists, const vmc_params *params,
                               vmc_walkers *walkers);

/*
 * ln|psi(n)| per walker (Sec. III.A): the Jastrow sum plus ln|det C^s_occ| of both spins, from
 * an FP64 LU of each C_occ block (no walker table is used or changed).  d_out: double [W].
 * A singular block gives -inf and latches VMC_ERR_SINGULAR.
 */
vmc_status vmc_log_psi(vmc_ctx *ctx, const vmc_walkers *walkers, const vmc_params *params,
                       double *d_out);

/*
 * Screened local energy, Eq. (eloc:hci), for every walker:
 *   E_L[n, eps_run] = e_diag + sum_{i->a kept} H ratio + sum_{ij->ab kept} H ratio
 * walking each occupied pair's sorted list up to the first |v| <= eps_run (eps_run >= the
 * build eps).  Ratios use G (Eq. R and its 2x2 minor) and the Jastrow sums.  The same ratios
 * are the CTMC rates r = |psi(m)/psi(n)| of Eq. (rate); their exact fixed-point sums are kept
 * in the context's rate store for vmc_ctmc_step, and the residence time t_n = 1/sum r is
 * returned.  d_e_loc, d_t_res: double [W] device outputs.
 */
vmc_status vmc_local_energy(vmc_ctx *ctx, const vmc_lists *lists, const vmc_params *params,
                            vmc_walkers *walkers, double eps_run, double *d_e_loc,
                            double *d_t_res);

/*
 * Continuous-time Monte Carlo move (Sec. II.B): for every walker pick the next determinant with
 * probability proportional to its rate, without rejection, from the rates stored by the last
 * vmc_local_energy on the same walkers (which must come first: VMC_ERR_ARG otherwise), then
 * update the walker in O(N^2): Sherman-Morrison (rank-1, or rank-2 Woodbury for same-spin
 * doubles) on G and AinvT, Jastrow sums, Fock sums, e_diag, bits and lists.
 * Choice rule: q_k = floor(r_k 2^64) (exact 128-bit), U = word 0 of
 * Philox4x64-10(key = (seed, walker index), counter = (rng_counter[w], 0, 0, 0)),
 * T = floor(U Q / 2^64) with Q = sum q_k; the first move in canonical order whose prefix sum
 * exceeds T is taken.  Canonical order: singles by (occupied spin orbital i ascending, list
 * position), then doubles by ((i,j) ascending lexicographically, list position).
 * d_move_code: uint64 [W] device output, kind | i<<2 | j<<12 | a<<22 | b<<32 (spin orbitals,
 * kind 1 = single with j = b = 1023, kind 2 = double).  rng_counter advances by one.
 */
vmc_status vmc_ctmc_step(vmc_ctx *ctx, const vmc_lists *lists, const vmc_params *params,
                         vmc_walkers *walkers, uint64_t seed, uint64_t *d_move_code);

/*
 * The screened move set of Sec. II.A / II.B for walkers w_begin .. w_begin + n_w - 1: every
 * determinant m connected to the walker's n by a single or double whose list entry survives
 * eps_run (>= the build eps) and whose target orbitals are empty -- the terms of E_L and the
 * moves of the CTMC step -- in the canonical order of vmc_ctmc_step.  For walker t of the range:
 *   d_code[t*cap + k]    uint64  move code as in vmc_ctmc_step
 *   d_ratio[t*cap + k]   double  psi(m)/psi(n) in the in-place replacement convention (the CTMC
 *                                rate is its magnitude; its sign differs from the canonically
 *                                ordered ratio by the permutation parity)
 *   d_contrib[t*cap + k] double  H_nm psi(m)/psi(n) (phase independent; sum + e_diag = E_L)
 *   d_count[t]           int64   number of moves of the walker (only the first cap are written)
 *   d_walked[2t], [2t+1] int64   singles and doubles list entries the walk reads, free or not
 *                                (NULL: not written)
 * The values are those vmc_local_energy and vmc_ctmc_step compute (same precision, same
 * rounding).  A diagnostic and test call: one warp walks each walker.  Calling it with another
 * eps_run than the last vmc_local_energy invalidates the stored rates (vmc_ctmc_step then
 * returns VMC_ERR_ARG until vmc_local_energy runs again).
 */
vmc_status vmc_screened_moves(vmc_ctx *ctx, const vmc_lists *lists, const vmc_params *params,
                              const vmc_walkers *walkers, double eps_run, int w_begin, int n_w,
                              int64_t cap, uint64_t *d_code, double *d_ratio, double *d_contrib,
                              int64_t *d_count, int64_t *d_walked);

/*
 * Batched launches over several systems of uneven size (for example Hubbard lattices and
 * hydrogen chains together).  Each item names one system's lists, parameters and walkers with
 * its own output arrays (d_e_loc, d_t_res: double [W]; d_move_code: uint64 [W]); all items must
 * use the same precision.  vmc_local_energy_batch computes every walker's local energy in one
 * launch whose CTAs stay resident and take walkers from a queue, most expensive systems first;
 * vmc_ctmc_step_batch then moves every walker (selection and update, one launch each).  Results
 * are identical to the per-system calls (walker index and seed as in vmc_ctmc_step).  The first
 * call with a new set of items uploads a small descriptor table (not capturable); later calls with
 * the same items are.  vmc_ctmc_step_batch must follow vmc_local_energy_batch on the same items.
 */
typedef struct {
    const vmc_lists *lists;
    const vmc_params *params;
    vmc_walkers *walkers;
    double eps_run;
    double *d_e_loc;
    double *d_t_res;
    uint64_t *d_move_code;
} vmc_batch_item;

vmc_status vmc_local_energy_batch(vmc_ctx *ctx, int n_items, const vmc_batch_item *items);
vmc_status vmc_ctmc_step_batch(vmc_ctx *ctx, int n_items, const vmc_batch_item *items, uint64_t seed);

/*
 * Autotuner for the local-energy launch: times 128, 256, 384 and 512 threads per walker CTA on the
 * given items (two launches each, CUDA events on the context's stream; vmc_local_energy for one
 * item, vmc_local_energy_batch for several), keeps the fastest for later vmc_local_energy /
 * vmc_local_energy_batch calls on this context and returns it.
 */
vmc_status vmc_autotune_local_energy(vmc_ctx *ctx, int n_items, const vmc_batch_item *items,
                                     int *threads_out);

/*
 * Vector-Jacobian product of ln psi (Sec. III.B gradient ratios) for weights w [W] (device):
 *   d_dJ[p][q]  += sum_w w_w n_p n_q   (p < q),   d_dJ[p][p] += sum_w w_w n_p   (upper triangle)
 *   d_dC_s[k][x] += sum_w w_w (C^s_occ)^-1[x][col(k)]   for occupied k of spin s
 * With w = t_n (E_L - E_ref) and w = t_n this gives the pieces of the energy gradient
 * g = 2 <(E_L - E) d ln psi/dp>, Eq. (grad).  Sums are FP64.
 */
vmc_status vmc_grad_logpsi(vmc_ctx *ctx, const vmc_walkers *walkers, const double *d_w,
                           double *d_dJ, double *d_dC_alpha, double *d_dC_beta);

/*
 * Correlator-product block of the vector-Jacobian product (Sec. III.B gradient ratios):
 *   d_dc[off_l + k] += sum_w w_w / c_l[k]   for the index k = n_l of every correlator l in walker w
 * (params->cps and walkers->cps_state required; d_dc: [n_values] FP64 device).  The sum is exact
 * in 64-bit fixed point before the final conversion, so it does not depend on summation order.
 */
vmc_status vmc_grad_logpsi_cps(vmc_ctx *ctx, const vmc_walkers *walkers, const vmc_params *params,
                               const double *d_w, double *d_dc);

/*
 * The two energy-gradient pieces of the correlator coefficients for one CTMC sweep (as
 * vmc_accumulate_gradient, whose walker sums d_sums it does not touch):
 *   d_AO_c += sum_w t_w d ln psi_w / dc,   d_AEO_c += sum_w t_w E_L,w d ln psi_w / dc.
 */
vmc_status vmc_accumulate_gradient_cps(vmc_ctx *ctx, const vmc_walkers *walkers, const vmc_params *params,
                                       const double *d_t_res, const double *d_e_loc, double *d_AO_c,
                                       double *d_AEO_c);

/*
 * Gradient accumulation for one CTMC sweep (Sec. II.B weights, Eq. grad pieces), one pass:
 *   d_sums[0] += sum_w t_w,  d_sums[1] += sum_w t_w E_L,w,
 *   A_O  += sum_w t_w d ln psi_w / dp,   A_EO += sum_w t_w E_L,w d ln psi_w / dp
 * for the walkers' current determinants (call after vmc_local_energy, before vmc_ctmc_step).
 * A_O and A_EO are each given as (dJ [(2M)^2], dC_alpha [M*na], dC_beta [M*nb]) device FP64
 * arrays laid out as in vmc_grad_logpsi.  d_t_res, d_e_loc: double [W].
 */
vmc_status vmc_accumulate_gradient(vmc_ctx *ctx, const vmc_walkers *walkers, const double *d_t_res,
                                   const double *d_e_loc, double *d_AO_J, double *d_AO_Ca,
                                   double *d_AO_Cb, double *d_AEO_J, double *d_AEO_Ca,
                                   double *d_AEO_Cb, double *d_sums);

/*
 * AMSGrad, Eqs. (m1)-(m2) as printed (beta1 weights the new gradient):
 *   m <- (1-beta1) m + beta1 g;  n <- max(n, (1-beta2) n + beta2 g^2);  p <- p - alpha m/sqrt(n)
 * with no update where n == 0.  All arrays FP64 device, length n_params.
 */
vmc_status vmc_amsgrad_update(vmc_ctx *ctx, double *d_p, const double *d_g, double *d_m,
                              double *d_n, size_t n_params, double alpha, double beta1,
                              double beta2);

/*
 * Energy gradient of Eq. (grad) from time-weighted sums over the samples of one iteration
 * (CTMC weights t_n, Sec. II.B):  with T = sums[0] = sum t and E = sums[1]/T,
 *   g_k = 2 (A_EO[k] / T - E * A_O[k] / T),   A_O = sum t O,  A_EO = sum t E_L O.
 * All device FP64 arrays of length n (g may alias neither input).  d_sums: double [2].
 */
vmc_status vmc_energy_gradient(vmc_ctx *ctx, size_t n, const double *d_sums, const double *d_A_O,
                               const double *d_A_EO, double *d_g);

/* Sum over walkers: out[0] += sum t, out[1] += sum t E_L (FP64, device out[2]). */
vmc_status vmc_walker_reduce(vmc_ctx *ctx, int W, const double *d_t_res, const double *d_e_loc,
                             double *d_out);

/*
 * vmc_grad_logpsi without any allocation and without a context (the paper has no counterpart;
 * it serves callers that may not allocate device memory: services whose device memory belongs to
 * another allocator's pool, deployments whose footprint is fixed up front, and host loops that
 * must not stall on the synchronisation cudaMalloc/cudaFree may cause).
 * Computes the same sums as vmc_grad_logpsi (accumulated into d_dJ, d_dC_alpha, d_dC_beta) for
 * weights d_w [W], using a library-owned 16 MiB device scratch array instead of a workspace.
 * Limit: 256 + 8 W (rounded up to 256 B) + max(32 M^2, 16 M n_max) bytes must fit in 16 MiB,
 * and 1 <= n_max <= 128 (n_max = max(n_alpha, n_beta)); otherwise VMC_ERR_ARG.  The first call on a device looks up the scratch
 * array's address (cudaGetSymbolAddress) with that device current: make it before any stream
 * capture.  All calls share the array: calls that overlap on the GPU race.  Work is queued on
 * `cuda_stream` (a cudaStream_t, NULL = legacy default stream).
 */
vmc_status vmc_grad_logpsi_noalloc(const vmc_walkers *walkers, const double *d_w, double *d_dJ,
                                   double *d_dC_alpha, double *d_dC_beta, void *cuda_stream);

/* Context options.  VMC_OPT_G_TENSOR_CORES (default 1): the refresh forms G = C C_occ^-1 on the
   tcgen05 tensor cores.  Mixed form: TF32 MMAs with a split-precision correction (0: FP32 CUDA
   cores).  FP64 form (register Gauss-Jordan refresh, n_sigma <= 128): every row of C and of
   C_occ^-T is scaled by a power of two and split into six BF16 digits of 8 bits, the digit
   products are summed exactly in FP32 and combined in 64-bit integers; G differs from the exact
   product by less than about 2^-43 n_sigma of the product of the two rows' power-of-two scales
   (0: FP64 FMAs on the CUDA cores).
   VMC_OPT_ELOC_THREADS: threads per local-energy CTA (128, 256, 384 or 512).
   VMC_OPT_MIXED_REFRESH_GJ32 (default 0): how VMC_MIXED recomputes C_occ^-1 at every refresh.
   0: LU with partial pivoting in FP64 in shared memory, the inverse from the factors and G in
   FP32 (the recompute is FP64, the tables FP32; n_sigma <= 128).  1: Gauss-Jordan elimination in
   FP32 with the matrix held in registers across a 16 x 16 thread grid (n_sigma <= 128), about
   4x faster on GB300, whose FP64 rate is 1/64 of its FP32 rate.
   VMC_OPT_REFRESH_SMEM (default 0): 1 replaces the register Gauss-Jordan kernels by the
   shared-memory kernels (mixed: the FP64 LU above; FP64: Gauss-Jordan with row exchanges,
   n_sigma <= 118); the FP64 form's default is the register Gauss-Jordan in FP64.
   VMC_OPT_GRAD_J_TENSOR_CORES (default 1): the Jastrow block of vmc_grad_logpsi and
   vmc_accumulate_gradient, sum_w c_w n_p n_q over walkers, runs as tcgen05 TF32 products of the
   0/1 occupation matrix with the eight base-256 digits of each 64-bit fixed-point weight (exact;
   0: the same fixed-point sums on the integer pipe).  Both give bit-identical results. */
#define VMC_OPT_G_TENSOR_CORES 1
#define VMC_OPT_ELOC_THREADS 2
#define VMC_OPT_REFRESH_SMEM 3
#define VMC_OPT_MIXED_REFRESH_GJ32 4
#define VMC_OPT_GRAD_J_TENSOR_CORES 5
vmc_status vmc_set_option(vmc_ctx *ctx, int option, int value);

/*
 * Measurement helper (no counterpart in the paper): one launch that reads the 16-byte-aligned
 * device buffer d_buf (bytes, a multiple of 16 is read) `reps` times with 16-byte loads through
 * L2, bypassing L1, on the context's stream.  Timed with events around it, for a buffer that fits
 * in L2 and after one warm-up call, bytes * reps / time is the L2 read bandwidth that bounds the
 * local energy's list traffic (the lists are shared by all walkers and stay in L2).
 */
vmc_status vmc_probe_l2_read(vmc_ctx *ctx, const void *d_buf, size_t bytes, int reps);

/* Number of kernel launches this context has issued (for accounting in benchmarks). */
uint64_t vmc_launch_count(const vmc_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* VMC_H */
