"""Seeded synthetic inputs: Hamiltonians, wavefunction parameters, initial determinants.

This module is shared by the CUDA path, the oracle and the tests.  It holds no arithmetic
of the VMC method itself (no local energy, ratio, sampling or optimisation step): it only
produces the integrals that define the Hamiltonian (Sec. II.A uses h_ij and <ab|ij>), the
parameters of the Jastrow-Slater wavefunction (Sec. III.A) and starting determinants.

Conventions used everywhere in this project
-------------------------------------------
* M spatial orbitals, 2M spin orbitals; spin orbital p = sigma*M + k (alpha block first).
* h1[p, q]                  one-electron integrals <p|h|q>, real symmetric, shape (M, M).
* eri[p, q, r, s] = (pq|rs) two-electron integrals in chemists' notation, shape (M,)*4,
  real orbitals, 8-fold symmetric.  The physicists' <pq|rs> of the paper is (pr|qs).
* e_core                    constant energy (nuclear repulsion), added to every E_L.
* J, shape (2M, 2M)         symmetric pair-Jastrow over spin orbitals; J[p, p] is the
  one-body term d_p.  ln C[n] = sum_{p<q} J_pq n_p n_q + sum_p J_pp n_p.
* C_alpha (M, n_alpha), C_beta (M, n_beta)  Slater coefficients theta of Sec. III.A.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy.special import erf

# STO-3G hydrogen 1s contraction (exponents, contraction coefficients).
STO3G_H_EXP = np.array([3.42525091, 0.62391373, 0.16885540])
STO3G_H_COEF = np.array([0.15432897, 0.53532814, 0.44463454])

MASTER_SEED = 1807


@dataclass
class System:
    """A Hamiltonian in an orthonormal orbital basis plus electron counts."""
    name: str
    M: int
    n_alpha: int
    n_beta: int
    h1: np.ndarray            # (M, M) float64
    eri: np.ndarray           # (M, M, M, M) float64, chemists' (pq|rs)
    e_core: float
    meta: dict = field(default_factory=dict)

    @property
    def n_elec(self) -> int:
        return self.n_alpha + self.n_beta


# ---------------------------------------------------------------------------------------
# Hubbard model (Sec. IV.C uses the 2-D Hubbard model; the 1-D ring is a small test case)
# ---------------------------------------------------------------------------------------
def hubbard(Lx: int, Ly: int = 1, t: float = 1.0, U: float = 4.0,
            n_alpha: int | None = None, n_beta: int | None = None) -> System:
    """Periodic Hubbard lattice: h_ij = -t for nearest neighbours, (ii|ii) = U."""
    M = Lx * Ly
    h1 = np.zeros((M, M))

    def site(x, y):
        return (y % Ly) * Lx + (x % Lx)

    for y in range(Ly):
        for x in range(Lx):
            s = site(x, y)
            nbrs = []
            if Lx > 1:
                nbrs += [site(x + 1, y), site(x - 1, y)]
            if Ly > 1:
                nbrs += [site(x, y + 1), site(x, y - 1)]
            for nb in set(nbrs):
                if nb != s:
                    h1[s, nb] = -t
    eri = np.zeros((M, M, M, M))
    for s in range(M):
        eri[s, s, s, s] = U
    na = M // 2 if n_alpha is None else n_alpha
    nb = M // 2 if n_beta is None else n_beta
    name = f"hubbard{Lx}" if Ly == 1 else f"hubbard{Lx}x{Ly}"
    return System(name, M, na, nb, h1, eri, 0.0, dict(t=t, U=U, Lx=Lx, Ly=Ly))


# ---------------------------------------------------------------------------------------
# Linear hydrogen chain, STO-3G, Loewdin-orthogonalised (local) orbitals
# ---------------------------------------------------------------------------------------
def _boys0(x: np.ndarray) -> np.ndarray:
    """Boys function F0(x) = 1/2 sqrt(pi/x) erf(sqrt(x)); series near 0."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    small = x < 1e-8
    xs = x[small]
    out[small] = 1.0 - xs / 3.0 + xs * xs / 10.0
    xl = x[~small]
    out[~small] = 0.5 * np.sqrt(np.pi / xl) * erf(np.sqrt(xl))
    return out


def _sgauss_ao_integrals(centers: np.ndarray, charges: np.ndarray, exps: np.ndarray,
                         coefs: np.ndarray, pair_cut: float = 1e-15, with_eri: bool = True):
    """Overlap S, core Hamiltonian h and ERIs (chemists') over contracted s-Gaussians.

    Closed forms for normalised s primitives (textbook Gaussian product theorem):
      S   = (pi/p)^{3/2} K_AB
      T   = ab/p (3 - 2 ab/p R_AB^2) (pi/p)^{3/2} K_AB
      V_C = -2 pi/p Z_C K_AB F0(p R_PC^2)
      ERI = 2 pi^{5/2} / (p q sqrt(p+q)) K_AB K_CD F0(p q/(p+q) R_PQ^2)
    with p = a+b, K_AB = exp(-ab/p R_AB^2), P = (aA+bB)/p.
    """
    nb = centers.shape[0]
    npr = exps.size
    norm = (2.0 * exps / np.pi) ** 0.75
    d = coefs * norm                                  # (npr,)
    # all primitive pairs of all AO pairs
    A = centers[:, None, None, None, :]
    B = centers[None, :, None, None, :]
    a = exps[None, None, :, None]
    b = exps[None, None, None, :]
    p = a + b
    R2 = np.sum((A - B) ** 2, axis=-1)                # (nb, nb, 1, 1)
    K = np.exp(-a * b / p * R2)
    P = (a[..., None] * A + b[..., None] * B) / p[..., None]   # (nb, nb, npr, npr, 3)
    dd = d[None, None, :, None] * d[None, None, None, :]
    S = np.sum(dd * (np.pi / p) ** 1.5 * K, axis=(2, 3))
    T = np.sum(dd * a * b / p * (3.0 - 2.0 * a * b / p * R2) * (np.pi / p) ** 1.5 * K,
               axis=(2, 3))
    V = np.zeros((nb, nb))
    for c in range(centers.shape[0]):
        RPC2 = np.sum((P - centers[c]) ** 2, axis=-1)
        V -= np.sum(dd * 2.0 * np.pi / p * charges[c] * K * _boys0(p * RPC2), axis=(2, 3))
    h = T + V
    if not with_eri:
        return S, h, None

    # ERIs: keep AO pairs (mu<=nu) whose pair prefactor is not negligible
    coef_pair = dd * K                                # (nb, nb, npr, npr)
    mu, nu = np.triu_indices(nb)
    keep = np.max(np.abs(coef_pair[mu, nu]).reshape(mu.size, -1), axis=1) > pair_cut
    mu, nu = mu[keep], nu[keep]
    npair = mu.size
    cp = coef_pair[mu, nu].reshape(npair, npr * npr)
    pp = np.broadcast_to(p, (nb, nb, npr, npr))[mu, nu].reshape(npair, npr * npr)
    PP = P[mu, nu].reshape(npair, npr * npr, 3)
    eri_pairs = np.zeros((npair, npair))
    chunk = max(1, 2_000_000 // (npair * npr ** 4) + 1)
    for i0 in range(0, npair, chunk):
        i1 = min(npair, i0 + chunk)
        pa = pp[i0:i1, None, :, None]                  # (c, 1, 9, 1)
        qa = pp[None, :, None, :]                      # (1, np, 1, 9)
        R2pq = np.sum((PP[i0:i1, None, :, None, :] - PP[None, :, None, :, :]) ** 2, axis=-1)
        pref = 2.0 * np.pi ** 2.5 / (pa * qa * np.sqrt(pa + qa))
        val = pref * _boys0(pa * qa / (pa + qa) * R2pq)
        val *= cp[i0:i1, None, :, None] * cp[None, :, None, :]
        eri_pairs[i0:i1] = val.sum(axis=(2, 3))
    eri = np.zeros((nb, nb, nb, nb))
    eri[mu[:, None], nu[:, None], mu[None, :], nu[None, :]] = eri_pairs
    eri[nu[:, None], mu[:, None], mu[None, :], nu[None, :]] = eri_pairs
    eri[mu[:, None], nu[:, None], nu[None, :], mu[None, :]] = eri_pairs
    eri[nu[:, None], mu[:, None], nu[None, :], mu[None, :]] = eri_pairs
    return S, h, eri


def pack_eri(eri: np.ndarray) -> np.ndarray:
    """Dense (pq|rs) [M^4] -> the 8-fold packed vector: pair index pq = p(p+1)/2 + q (p >= q),
    element PQ(PQ+1)/2 + RS (PQ >= RS); each element is taken from (pq|rs) with p >= q, r >= s,
    PQ >= RS.  A storage format only (M(M+1)/2 (M(M+1)/2 + 1)/2 doubles)."""
    M = eri.shape[0]
    p, q = np.tril_indices(M)                      # pair PQ = p(p+1)/2 + q in this order
    P, R = np.tril_indices(p.size)
    return np.ascontiguousarray(eri[p[P], q[P], p[R], q[R]])


def unpack_eri(packed: np.ndarray, M: int) -> np.ndarray:
    """The 8-fold packed vector of pack_eri -> a dense, exactly 8-fold symmetric [M^4] array."""
    p, q = np.tril_indices(M)
    npair = p.size
    pair = np.zeros((M, M), dtype=np.int64)
    pair[p, q] = np.arange(npair)
    pair[q, p] = np.arange(npair)
    RS = pair.reshape(-1)
    out = np.empty((M, M, M, M))
    for a in range(M):                             # one bra orbital at a time: O(M^3) indices
        PQ = pair[a][:, None]
        A, B = np.maximum(PQ, RS[None, :]), np.minimum(PQ, RS[None, :])
        out[a] = packed[A * (A + 1) // 2 + B].reshape(M, M, M)
    return out


def _transform_eri(eri: np.ndarray, X: np.ndarray) -> np.ndarray:
    """(pq|rs) <- sum X[mu,p] X[nu,q] X[la,r] X[si,s] (mu nu|la si).

    Ket pair first (batched X^T E X over the M^2 bra rows), then the bra pair (one matmul on
    the leading axis and one batched over it); no large transposes are made.  Uses torch's
    multithreaded CPU matmul (input preparation only)."""
    import torch

    M = X.shape[0]
    E = torch.from_numpy(np.ascontiguousarray(eri))
    Xt = torch.from_numpy(np.ascontiguousarray(X))
    Y = torch.matmul(torch.matmul(Xt.T, E.reshape(M * M, M, M)), Xt)     # (M^2, M, M)
    T1 = (Xt.T @ Y.reshape(M, M * M * M)).reshape(M, M, M * M)
    del Y
    R = torch.matmul(Xt.T, T1)                                            # (M, M, M^2)
    return R.reshape(M, M, M, M).numpy()


def _chain_ao_eri(n_atoms: int, spacing: float, exps: np.ndarray, coefs: np.ndarray,
                  pair_cut: float = 1e-15) -> np.ndarray:
    """AO ERIs of a uniform linear chain of identical s shells.

    (mu nu|la si) with mu <= nu, la <= si depends only on d = nu - mu, e = si - la and the
    offset la - mu, so a table over (d, e, offset) is evaluated once and gathered."""
    npr = exps.size
    d_norm = coefs * (2.0 * exps / np.pi) ** 0.75
    a = exps[:, None]
    b = exps[None, :]
    p = a + b
    dd = d_norm[:, None] * d_norm[None, :]
    # largest pair length whose primitive prefactors are not negligible
    D = 0
    while D + 1 < n_atoms and np.max(np.abs(dd * np.exp(-a * b / p * (spacing * (D + 1)) ** 2))) > pair_cut:
        D += 1
    dists = np.arange(D + 1)
    K = np.exp(-a[None] * b[None] / p[None] * (spacing * dists[:, None, None]) ** 2)   # (D+1, npr, npr)
    cpair = (dd[None] * K).reshape(D + 1, -1)                                       # (D+1, 9)
    shift = (b[None] * spacing * dists[:, None, None] / p[None]).reshape(D + 1, -1)  # P - A
    pp = np.broadcast_to(p, (npr, npr)).reshape(-1)
    offs = np.arange(-(n_atoms - 1), n_atoms)
    # table[d, e, o]: pair (0, d) against pair (o, o + e)
    Pd = shift[:, None, None, :, None]                                     # (D+1,1,1,9,1)
    Qe = spacing * offs[None, None, :, None, None] + shift[None, :, None, None, :]   # (1,D+1,O,1,9)
    R2 = (Pd - Qe) ** 2
    pa = pp[None, None, None, :, None]
    qa = pp[None, None, None, None, :]
    val = 2.0 * np.pi ** 2.5 / (pa * qa * np.sqrt(pa + qa)) * _boys0(pa * qa / (pa + qa) * R2)
    val *= cpair[:, None, None, :, None] * cpair[None, :, None, None, :]
    table = val.sum(axis=(3, 4))                                           # (D+1, D+1, O)
    mu = np.concatenate([np.arange(n_atoms - d) for d in dists])
    dl = np.concatenate([np.full(n_atoms - d, d) for d in dists])
    nu = mu + dl
    ep = table[dl[:, None], dl[None, :], (mu[None, :] - mu[:, None]) + (n_atoms - 1)]
    M = n_atoms
    eri = np.zeros((M, M, M, M))
    eri[mu[:, None], nu[:, None], mu[None, :], nu[None, :]] = ep
    eri[nu[:, None], mu[:, None], mu[None, :], nu[None, :]] = ep
    eri[mu[:, None], nu[:, None], nu[None, :], mu[None, :]] = ep
    eri[nu[:, None], mu[:, None], nu[None, :], mu[None, :]] = ep
    return eri


def hchain(n_atoms: int, spacing: float = 1.8) -> System:
    """Linear H_n chain in STO-3G, integrals in Loewdin-orthogonalised AOs (local orbitals)."""
    centers = np.zeros((n_atoms, 3))
    centers[:, 0] = spacing * np.arange(n_atoms)
    charges = np.ones(n_atoms)
    S, h, _ = _sgauss_ao_integrals(centers, charges, STO3G_H_EXP, STO3G_H_COEF, with_eri=False)
    eri_ao = _chain_ao_eri(n_atoms, spacing, STO3G_H_EXP, STO3G_H_COEF)
    s, U = np.linalg.eigh(S)
    X = (U * s ** -0.5) @ U.T                          # S^{-1/2}, symmetric
    h1 = X.T @ h @ X
    h1 = 0.5 * (h1 + h1.T)
    eri = _transform_eri(eri_ao, X)
    del eri_ao
    # the transform leaves (pq|rs) and its symmetric images a few ulps apart; keep one value per
    # symmetry class so the integrals are exactly 8-fold symmetric (dense and packed input agree)
    eri = unpack_eri(pack_eri(eri), n_atoms)
    e_core = 0.0
    for A in range(n_atoms):
        for B in range(A + 1, n_atoms):
            e_core += 1.0 / (spacing * (B - A))
    na = (n_atoms + 1) // 2
    nb = n_atoms // 2
    return System(f"H{n_atoms}", n_atoms, na, nb, h1, eri, e_core,
                  dict(spacing=spacing, basis="sto-3g", orbitals="lowdin"))


# ---------------------------------------------------------------------------------------
# Wavefunction parameters (Sec. III.A; pair Jastrow = two-site correlators)
# ---------------------------------------------------------------------------------------
@dataclass
class Params:
    J: np.ndarray            # (2M, 2M) symmetric; diagonal = one-body terms
    C_alpha: np.ndarray      # (M, n_alpha)
    C_beta: np.ndarray       # (M, n_beta)

    def flat(self) -> np.ndarray:
        return np.concatenate([self.J.ravel(), self.C_alpha.ravel(), self.C_beta.ravel()])


def random_jastrow(M: int, rng: np.random.Generator, scale: float = 0.01) -> np.ndarray:
    A = rng.normal(0.0, scale, size=(2 * M, 2 * M))
    J = np.triu(A) + np.triu(A, 1).T
    return J


def planewave_ring(L: int, n: int) -> np.ndarray:
    """Real plane waves on a ring: 1, cos(2 pi k x/L), sin(2 pi k x/L), k = 1, 2, ..."""
    x = np.arange(L)
    cols = [np.ones(L)]
    k = 1
    while len(cols) < n:
        cols.append(np.cos(2 * np.pi * k * x / L))
        if len(cols) < n:
            cols.append(np.sin(2 * np.pi * k * x / L))
        k += 1
    C = np.stack(cols, axis=1)
    return C / np.linalg.norm(C, axis=0)


def core_orbitals(h1: np.ndarray, n: int) -> np.ndarray:
    """Lowest n eigenvectors of h1 (core-Hamiltonian guess), sign-fixed."""
    _, V = np.linalg.eigh(h1)
    V = V[:, :n].copy()
    for c in range(n):
        if V[np.argmax(np.abs(V[:, c])), c] < 0:
            V[:, c] *= -1
    return V


def neel_orbitals(M: int, n: int, offset: int) -> np.ndarray:
    """Local orbitals on alternating sites offset, offset + 2, ... (n columns of the identity): the
    antiferromagnetic determinant of a stretched chain in local orbitals, alpha on even sites and
    beta on odd ones, the shape a broken-symmetry (unrestricted) mean-field solution takes there."""
    sites = [(offset + 2 * k) % M for k in range(n)]
    if len(set(sites)) != n:
        raise ValueError("more electrons of one spin than alternating sites")
    C = np.zeros((M, n))
    C[sites, np.arange(n)] = 1.0
    return C


def make_params(sys: System, seed: int = MASTER_SEED, j_scale: float = 0.01,
                c_noise: float = 0.01, zero_jastrow: bool = False,
                exact_planewave: bool = False, start: str = "core") -> Params:
    """Seeded Jastrow-Slater parameters.

    Slater part: Hubbard rings use real plane waves, everything else the core-Hamiltonian
    orbitals (start="core") or the alternating-site determinant (start="neel"); both get an
    independent N(0, c_noise) perturbation per spin (unrestricted).
    Jastrow: J ~ N(0, j_scale), symmetric, over spin-orbital pairs.
    """
    rng = np.random.default_rng(seed)
    M = sys.M
    J = np.zeros((2 * M, 2 * M)) if zero_jastrow else random_jastrow(M, rng, j_scale)
    if sys.name.startswith("hubbard") and sys.meta.get("Ly", 1) == 1:
        Ca = planewave_ring(M, sys.n_alpha)
        Cb = planewave_ring(M, sys.n_beta)
    elif start == "neel":
        Ca = neel_orbitals(M, sys.n_alpha, 0)
        Cb = neel_orbitals(M, sys.n_beta, 1)
    else:
        Ca = core_orbitals(sys.h1, sys.n_alpha)
        Cb = core_orbitals(sys.h1, sys.n_beta)
    if not exact_planewave:
        Ca = Ca + rng.normal(0.0, c_noise, size=Ca.shape)
        Cb = Cb + rng.normal(0.0, c_noise, size=Cb.shape)
    return Params(J, np.ascontiguousarray(Ca), np.ascontiguousarray(Cb))


# ---------------------------------------------------------------------------------------
# Starting determinants (the paper is silent)
# ---------------------------------------------------------------------------------------
# ---------------------------------------------------------------------------------------
# Correlator product (Sec. III.A): local correlators of at most five sites, one centred on every
# site (Sec. IV.B-C).  The pair Jastrow above is the special case of one- and two-site correlators.
# ---------------------------------------------------------------------------------------
@dataclass
class CPS:
    """Correlator l covers the spatial sites ``sites[l]`` and holds ``4 ** len(sites[l])``
    coefficients ``values[l]``, indexed by sum_t (n_alpha(site_t) + 2 n_beta(site_t)) 4**t."""
    sites: list
    values: list


def correlator_sites(sys: System, size: int = 5) -> list:
    """Sites of the local correlator centred on each site: on a chain the `size` consecutive
    sites around it (clipped at the ends), on a ring the same with periodic wrap, on a 2-D
    lattice the site and its four neighbours."""
    M = sys.M
    Lx, Ly = sys.meta.get("Lx"), sys.meta.get("Ly")
    h = size // 2
    out = []
    for c in range(M):
        if Lx is not None and Ly is not None and Ly > 1:
            x, y = c % Lx, c // Lx
            cand = [c, y * Lx + (x + 1) % Lx, y * Lx + (x - 1) % Lx, ((y + 1) % Ly) * Lx + x,
                    ((y - 1) % Ly) * Lx + x]
        elif Lx is not None:
            cand = [(c + d) % M for d in range(-h, h + 1)]
        else:
            cand = list(range(max(0, c - h), min(M, c + h + 1)))
        sites = []
        for q in cand:
            if q not in sites:
                sites.append(q)
        out.append(np.array(sites, dtype=np.int32))
    return out


def make_cps(sys: System, size: int = 5, seed: int = MASTER_SEED, noise: float = 0.05) -> CPS:
    """Seeded correlator coefficients 1 + noise * N(0, 1) on the local correlators."""
    rng = np.random.default_rng(seed)
    sites = correlator_sites(sys, size)
    values = [1.0 + noise * rng.normal(size=4 ** len(st)) for st in sites]
    return CPS(sites, values)


def _dpp_rows(C: np.ndarray, B: int, rng: np.random.Generator) -> np.ndarray:
    """B independent draws of n rows of C (M x n) with probability proportional to
    det(C[rows])^2: sequential sampling of the projection determinantal point process onto the
    column space of C (Hough, Krishnapur, Peres & Virag, 2006).  Returns (B, n) sorted rows.

    With Q an orthonormal basis of the column space, row m is drawn at step k with probability
    proportional to its squared distance from the span of the rows already drawn; the basis u_t of
    that span is grown by Gram-Schmidt (twice, for orthogonality) and the distances are updated by
    the projections Q u_k (batched over the B draws with torch's CPU matmul)."""
    import torch

    M, n = C.shape
    Q, _ = np.linalg.qr(C)                          # orthonormal basis of the column space
    Qt = torch.from_numpy(np.ascontiguousarray(Q))
    r = torch.from_numpy(np.broadcast_to(np.sum(Q * Q, axis=1), (B, M)).copy())   # squared distances
    U = torch.zeros((B, n, n), dtype=torch.float64)
    rows = np.empty((B, n), dtype=np.int64)
    ar = torch.arange(B)
    for k in range(n):
        p = torch.clamp(r, min=0.0)
        p /= p.sum(dim=1, keepdim=True)
        u = torch.from_numpy(rng.random(B))[:, None]
        i = torch.clamp((torch.cumsum(p, dim=1) < u).sum(dim=1), max=M - 1)
        rows[:, k] = i.numpy()
        v = Qt[i].clone()
        if k:
            Uk = U[:, :k]
            for _ in range(2):
                v -= torch.bmm(Uk.transpose(1, 2), torch.bmm(Uk, v[:, :, None]))[:, :, 0]
        v /= torch.linalg.norm(v, dim=1, keepdim=True)
        U[:, k] = v
        proj = v @ Qt.T
        r -= proj * proj
        r[ar, i] = 0.0
    return np.sort(rows, axis=1)


def init_occupations(sys: System, prm: Params, W: int, seed: int = MASTER_SEED + 1,
                     chunk: int = 512) -> np.ndarray:
    """Per-walker occupied orbital lists, shape (W, n_alpha + n_beta), uint16, each spin block
    sorted ascending (alpha orbitals, then beta; spatial indices 0..M-1).

    Each spin's orbitals are an exact draw from |det C^s[rows]|^2, the distribution the Slater
    part alone would be sampled from, so walkers start at typical, well-conditioned
    determinants.  Every walker gets its own draw."""
    rng = np.random.default_rng(seed)
    na, nb = sys.n_alpha, sys.n_beta
    occ = np.empty((W, na + nb), dtype=np.uint16)
    for c0 in range(0, W, chunk):
        c1 = min(W, c0 + chunk)
        if na:
            occ[c0:c1, :na] = _dpp_rows(prm.C_alpha, c1 - c0, rng)
        if nb:
            occ[c0:c1, na:] = _dpp_rows(prm.C_beta, c1 - c0, rng)
    return occ


def occ_to_bits(occ: np.ndarray, M: int, n_alpha: int) -> np.ndarray:
    """(W, n_e) occupied lists -> (W, 2, ceil(M/32)) uint32 bitstrings per spin."""
    W = occ.shape[0]
    nw = (M + 31) // 32
    bits = np.zeros((W, 2, nw), dtype=np.uint32)
    for w in range(W):
        for c, k in enumerate(occ[w]):
            s = 0 if c < n_alpha else 1
            bits[w, s, int(k) // 32] |= np.uint32(1 << (int(k) % 32))
    return bits


def named_system(name: str) -> System:
    """Workloads by name: 'hubbard10', 'hubbard4x4', 'H20', ..."""
    if name.startswith("hubbard"):
        dims = name[len("hubbard"):]
        if "x" in dims:
            lx, ly = (int(v) for v in dims.split("x"))
            return hubbard(lx, ly, t=1.0, U=4.0)
        return hubbard(int(dims), 1, t=1.0, U=4.0)
    if name.startswith("H"):
        return hchain(int(name[1:]))
    raise ValueError(name)
