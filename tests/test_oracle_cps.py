"""Pins for the oracle's correlator product (CPS) of Sec. III.A, the wavefunction of the paper's
benchmarks: psi(n) = prod_l c_l[n_l] x det theta_alpha[n] x det theta_beta[n] (times the pair
Jastrow when it is non-zero).  Each test ties the oracle to something other than itself: brute
force over every determinant, the already pinned pair-Jastrow path, finite differences and the
exact energy.  CPU only."""
import math

import numpy as np
import pytest

import oracle
from oracle import Oracle
from paper_1807_10633_gb300 import systems as S
from tests import brute


def _case(sys_, seed=5, noise=0.2, j_scale=0.0):
    prm = S.make_params(sys_, seed=seed, j_scale=j_scale, c_noise=0.1)
    if j_scale == 0.0:
        prm.J[:] = 0.0
    return prm, S.make_cps(sys_, seed=seed + 1, noise=noise)


@pytest.mark.parametrize("make", [lambda: S.hchain(4), lambda: S.hchain(6), lambda: S.hubbard(10, 1),
                                  lambda: S.hubbard(3, 3)], ids=["H4", "H6", "ring10", "lattice3x3"])
def test_cps_eloc_eps0_matches_brute_all_dets(make):
    """E_L at eps = 0 equals (H psi)(n)/psi(n) for every determinant, with 5-site correlators
    (clipped windows on a chain, periodic windows on a ring, plus shapes on a lattice) and a
    non-zero pair Jastrow on top."""
    sys_ = make()
    prm, cps = _case(sys_, j_scale=0.05)
    dets, H = brute.hamiltonian(sys_)
    n = brute.occupations(dets, sys_.M)
    psi = brute.psi_all(n, sys_.M, prm) * brute.cps_factor(n, sys_.M, cps)
    el, _, _ = Oracle(sys_, prm, cps).local_energy_batch(n, 0.0)
    np.testing.assert_allclose(el, (H @ psi) / psi, rtol=1e-10, atol=1e-10)


def _jastrow_as_cps(J, M):
    """The pair Jastrow written as one- and two-site correlators: site p carries the terms of
    J among p_alpha and p_beta, the pair (p, q) the four cross terms."""
    sites, vals = [], []
    for p in range(M):
        a, b = p, M + p
        v = np.zeros(4)
        for st in range(4):
            na, nb = st & 1, st >> 1
            v[st] = math.exp(J[a, a] * na + J[b, b] * nb + J[a, b] * na * nb)
        sites.append(np.array([p], dtype=np.int32)); vals.append(v)
    for p in range(M):
        for q in range(p + 1, M):
            v = np.zeros(16)
            for st in range(16):
                npa, npb, nqa, nqb = st & 1, (st >> 1) & 1, (st >> 2) & 1, (st >> 3) & 1
                x = (J[p, q] * npa * nqa + J[p, M + q] * npa * nqb + J[q, M + p] * npb * nqa
                     + J[M + p, M + q] * npb * nqb)        # upper-triangle entries (row < column)
                v[st] = math.exp(x)
            sites.append(np.array([p, q], dtype=np.int32)); vals.append(v)
    return S.CPS(sites, vals)


def test_pair_jastrow_written_as_correlators_gives_the_same_energies():
    """The CPS path with one- and two-site correlators built from J reproduces the pinned
    pair-Jastrow path exactly (this fixes which bit of a site is alpha and which digit is which
    site, independently of the brute-force factor)."""
    sys_ = S.hchain(6)
    prm = S.make_params(sys_, seed=13, j_scale=0.2, c_noise=0.1)
    J = np.triu(prm.J)                       # the Jastrow reads its upper triangle
    cps = _jastrow_as_cps(J, sys_.M)
    zero = S.Params(np.zeros_like(prm.J), prm.C_alpha, prm.C_beta)
    n = brute.occupations(brute.all_dets(sys_.M, sys_.n_alpha, sys_.n_beta), sys_.M)
    e_j, _, _ = Oracle(sys_, prm).local_energy_batch(n, 1e-6)
    e_c, _, _ = Oracle(sys_, zero, cps).local_energy_batch(n, 1e-6)
    np.testing.assert_allclose(e_c, e_j, rtol=1e-12, atol=1e-12)
    o1, o2 = Oracle(sys_, prm), Oracle(sys_, zero, cps)
    for d in (0, 17, 123, 399):
        assert abs(o2.psi(n[d]) - o1.psi(n[d])) <= 1e-13 * abs(o1.psi(n[d]))


def test_cps_gradient_matches_finite_differences():
    """d ln psi / d c_l[k] = delta(k, n_l) / c_l[k] against central differences of the brute
    ln|psi| for every coefficient of three correlators (active ones and zeros)."""
    sys_ = S.hchain(6)
    prm, cps = _case(sys_, seed=8, j_scale=0.05)
    orc = Oracle(sys_, prm, cps)
    n = brute.occupations(brute.all_dets(sys_.M, 3, 3), sys_.M)[[123]]
    dc = np.zeros(orc.n_corr_values)
    orc.grad_cps(n[0], 1.0, dc)
    off = np.concatenate([[0], np.cumsum([len(v) for v in cps.values])])

    def lnpsi(c):
        return math.log(abs(brute.psi_all(n, sys_.M, prm)[0] * brute.cps_factor(n, sys_.M, c)[0]))

    h = 1e-6
    for l in (0, 2, 5):
        for k in range(len(cps.values[l])):
            vp = [v.copy() for v in cps.values]
            vm = [v.copy() for v in cps.values]
            vp[l][k] += h
            vm[l][k] -= h
            fd = (lnpsi(S.CPS(cps.sites, vp)) - lnpsi(S.CPS(cps.sites, vm))) / (2 * h)
            assert abs(fd - dc[off[l] + k]) < 1e-7 * max(1.0, abs(fd)), (l, k)
    assert np.count_nonzero(dc) == len(cps.sites)      # one active coefficient per correlator


def test_cps_energy_gradient_matches_exact_derivative():
    """2 <(E_L - E) O_c>_rho (Eq. grad, with the oracle's E_L and d ln psi / d c) equals the
    derivative of the exact energy <psi|H|psi>/<psi|psi> with respect to a coefficient."""
    sys_ = S.hubbard(6, 1)
    prm, cps = _case(sys_, seed=4, j_scale=0.05)
    dets, H = brute.hamiltonian(sys_)
    n = brute.occupations(dets, sys_.M)

    def energy(c):
        psi = brute.psi_all(n, sys_.M, prm) * brute.cps_factor(n, sys_.M, c)
        return float(psi @ (H @ psi) / (psi @ psi))

    orc = Oracle(sys_, prm, cps)
    el, _, _ = orc.local_energy_batch(n, 0.0)
    psi = brute.psi_all(n, sys_.M, prm) * brute.cps_factor(n, sys_.M, cps)
    rho = psi ** 2 / np.sum(psi ** 2)
    E = float(rho @ el)
    g = np.zeros(orc.n_corr_values)
    for d in range(len(n)):
        orc.grad_cps(n[d], 2.0 * rho[d] * (el[d] - E), g)
    off = np.concatenate([[0], np.cumsum([len(v) for v in cps.values])])
    h = 1e-5
    rng = np.random.default_rng(9)
    for _ in range(6):
        l = int(rng.integers(len(cps.sites)))
        k = int(np.argmax(np.abs(g[off[l]:off[l + 1]])))
        vp = [v.copy() for v in cps.values]
        vm = [v.copy() for v in cps.values]
        vp[l][k] += h
        vm[l][k] -= h
        fd = (energy(S.CPS(cps.sites, vp)) - energy(S.CPS(cps.sites, vm))) / (2 * h)
        assert abs(fd - g[off[l] + k]) < 1e-6 * max(1.0, abs(fd)), (l, k, fd, g[off[l] + k])


def test_correlator_sites_follow_the_lattice():
    chain = S.correlator_sites(S.hchain(8))
    assert [list(x) for x in chain[:3]] == [[0, 1, 2], [0, 1, 2, 3], [0, 1, 2, 3, 4]]
    assert list(chain[7]) == [5, 6, 7]
    ring = S.correlator_sites(S.hubbard(8, 1))
    assert sorted(ring[0]) == [0, 1, 2, 6, 7] and all(len(x) == 5 for x in ring)
    lat = S.correlator_sites(S.hubbard(4, 4))
    assert sorted(lat[5]) == [1, 4, 5, 6, 9] and all(len(x) == 5 for x in lat)
    assert sorted(lat[0]) == [0, 1, 3, 4, 12]             # periodic neighbours


def test_cps_move_ratios_are_brute_force_psi_ratios():
    """Every screened move's psi(m)/psi(n) -- the CTMC rate up to its sign (Sec. II.B) -- equals
    the ratio of the brute-force amplitudes with correlators, so the rates and the residence time
    of a CPS-Slater walker follow from the same ratios as its local energy."""
    sys_ = S.hchain(6)
    prm, cps = _case(sys_, seed=31, j_scale=0.05)
    dets, _ = brute.hamiltonian(sys_)
    n_all = brute.occupations(dets, sys_.M)
    psi = brute.psi_all(n_all, sys_.M, prm) * brute.cps_factor(n_all, sys_.M, cps)
    weights = np.arange(2 * sys_.M, dtype=np.uint64)
    orc = Oracle(sys_, prm, cps)
    rng = np.random.default_rng(5)
    checked = 0
    for d in rng.choice(len(n_all), 10, replace=False):
        n = n_all[d]
        _, _, mv = orc.local_energy(n, 1e-4)
        for o in mv:
            m = n.copy()
            m[o["i"]] = 0
            m[o["a"]] = 1
            if o["kind"] == 2:
                m[o["j"]] = 0
                m[o["b"]] = 1
            idx = np.searchsorted(dets, (m.astype(np.uint64) << weights).sum())
            ref = psi[idx] / psi[d]
            assert abs(o["ratio"] - ref) <= 1e-11 * max(1.0, abs(ref))
            checked += 1
    assert checked > 500
