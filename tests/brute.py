"""Brute-force reference over the full determinant space (tiny systems only).

Independent of the oracle: the Hamiltonian matrix is built by applying the second-quantised
operators  H = sum_pq h_pq a+_p a_q + 1/2 sum_pqrs <pq|rs> a+_p a+_q a_s a_r  (+ E_core)
to every determinant (bit masks, vectorised with numpy), and psi(n) is evaluated from its
definition (Jastrow sum and two numpy determinants).  Used to pin the oracle.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp


def all_dets(M: int, na: int, nb: int) -> np.ndarray:
    """Sorted uint64 bit masks (bit p = spin orbital p occupied, p = sigma*M + k)."""
    A = [sum(1 << k for k in c) for c in itertools.combinations(range(M), na)]
    B = [sum(1 << (M + k) for k in c) for c in itertools.combinations(range(M), nb)]
    masks = np.array([a | b for a in A for b in B], dtype=np.uint64)
    return np.sort(masks)


def _apply(masks, phase, valid, p, create):
    bit = np.uint64(1) << np.uint64(p)
    occ = (masks & bit) != 0
    ok = valid & (~occ if create else occ)
    below = masks & (bit - np.uint64(1))
    par = np.bitwise_count(below) & 1
    phase = np.where(par == 1, -phase, phase)
    return masks ^ np.where(ok, bit, np.uint64(0)), phase, ok


def hamiltonian(sys) -> tuple[np.ndarray, sp.csr_matrix]:
    M = sys.M
    dets = all_dets(M, sys.n_alpha, sys.n_beta)
    nd = dets.size
    rows, cols, vals = [], [], []

    def add_term(coef, ops):
        # ops applied right to left: list of (p, create)
        m = dets.copy()
        ph = np.ones(nd)
        ok = np.ones(nd, dtype=bool)
        for p, cr in reversed(ops):
            m, ph, ok = _apply(m, ph, ok, p, cr)
        idx = np.searchsorted(dets, m)
        idx = np.minimum(idx, nd - 1)
        ok &= dets[idx] == m
        rows.append(idx[ok])
        cols.append(np.nonzero(ok)[0])
        vals.append(coef * ph[ok])

    N2 = 2 * M
    spin = lambda p: p // M
    sp_ = lambda p: p % M
    for p in range(N2):
        for q in range(N2):
            if spin(p) != spin(q):
                continue
            h = sys.h1[sp_(p), sp_(q)]
            if h != 0.0:
                add_term(h, [(p, True), (q, False)])
    for p, q, r, s in itertools.product(range(N2), repeat=4):
        if spin(p) != spin(r) or spin(q) != spin(s):
            continue
        v = sys.eri[sp_(p), sp_(r), sp_(q), sp_(s)]      # <pq|rs> = (pr|qs)
        if v == 0.0 or p == q or r == s:
            continue
        add_term(0.5 * v, [(p, True), (q, True), (s, False), (r, False)])
    H = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(nd, nd)).tocsr()
    H = H + sys.e_core * sp.identity(nd, format="csr")
    return dets, H


def occupations(dets: np.ndarray, M: int) -> np.ndarray:
    """(nd, 2M) uint8 occupation numbers."""
    p = np.arange(2 * M, dtype=np.uint64)
    return ((dets[:, None] >> p[None, :]) & np.uint64(1)).astype(np.uint8)


def psi_all(n: np.ndarray, M: int, prm) -> np.ndarray:
    """psi(n) = exp(sum_{p<q} J_pq n_p n_q + sum_p J_pp n_p) det Ca[occ_a] det Cb[occ_b]."""
    Ju = np.triu(prm.J)
    nf = n.astype(np.float64)
    lnC = np.einsum("dp,pq,dq->d", nf, Ju, nf)
    na = prm.C_alpha.shape[1]
    nb = prm.C_beta.shape[1]
    occa = np.array([np.nonzero(r[:M])[0] for r in n])
    occb = np.array([np.nonzero(r[M:])[0] for r in n])
    da = np.linalg.det(prm.C_alpha[occa]) if na else np.ones(len(n))
    db = np.linalg.det(prm.C_beta[occb]) if nb else np.ones(len(n))
    return np.exp(lnC) * da * db


def cps_factor(n: np.ndarray, M: int, cps) -> np.ndarray:
    """prod over correlators of c_l[state of its sites], each site's state n_alpha + 2 n_beta read
    as a base-4 digit (first site least significant)."""
    out = np.ones(len(n))
    for sites, vals in zip(cps.sites, cps.values):
        idx = np.zeros(len(n), dtype=np.int64)
        for t, site in enumerate(sites):
            idx += (4 ** t) * (n[:, site].astype(np.int64) + 2 * n[:, M + site].astype(np.int64))
        out *= np.asarray(vals)[idx]
    return out


def singles_bound(sys) -> np.ndarray:
    """S_ia over spatial orbitals (spin independent): |h_ia| + sum over all spin orbitals j."""
    e = sys.eri
    Jt = np.einsum("iakk->iak", e)       # <ij|aj> = (ia|jj) for every j
    Kt = np.einsum("ikka->iak", e)       # <ij|ja> = (ij|ja) for same-spin j
    return np.abs(sys.h1) + np.abs(Jt - Kt).sum(-1) + np.abs(Jt).sum(-1)
