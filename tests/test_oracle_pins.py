"""Pins for the oracle: each test ties it to something other than itself.

Brute force over the full determinant space (tests/brute.py builds H from second-quantised
operators), closed forms, library routines (numpy's Philox, scipy's eigsh) and finite
differences.  CPU only.
"""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as sla

import oracle
from oracle import Oracle, occ_lists_to_n
from paper_1807_10633_gb300 import systems as S
from tests import brute


def _h4():
    return S.hchain(4)


def _h6():
    return S.hchain(6)


@pytest.fixture(scope="module")
def hub10():
    sys = S.hubbard(10, 1, t=1.0, U=4.0)
    prm = S.make_params(sys, seed=11)
    dets, H = brute.hamiltonian(sys)
    n = brute.occupations(dets, sys.M)
    psi = brute.psi_all(n, sys.M, prm)
    return sys, prm, dets, H, n, psi


def _brute_eloc(H, psi):
    return (H @ psi) / psi


# --- E_L at eps = 0 equals (H psi)(n) / psi(n) for every determinant (Sec. II.A) ---------
def test_eloc_eps0_matches_brute_hubbard10_all_dets(hub10):
    sys, prm, dets, H, n, psi = hub10
    orc = Oracle(sys, prm)
    el, _, _ = orc.local_energy_batch(n, 0.0)
    ref = _brute_eloc(H, psi)
    np.testing.assert_allclose(el, ref, rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("make", [_h4, _h6])
def test_eloc_eps0_matches_brute_hchain(make):
    sys = make()
    prm = S.make_params(sys, seed=5, j_scale=0.05, c_noise=0.1)
    dets, H = brute.hamiltonian(sys)
    n = brute.occupations(dets, sys.M)
    psi = brute.psi_all(n, sys.M, prm)
    orc = Oracle(sys, prm)
    el, _, _ = orc.local_energy_batch(n, 0.0)
    np.testing.assert_allclose(el, _brute_eloc(H, psi), rtol=1e-10, atol=1e-10)


# --- direct determinant ratios equal the G-table ratios (Eq. R and its 2x2 minor) --------
def test_direct_ratios_equal_table_ratios():
    sys = _h6()
    prm = S.make_params(sys, seed=9, j_scale=0.1, c_noise=0.2)
    orc = Oracle(sys, prm)
    dets = brute.all_dets(sys.M, sys.n_alpha, sys.n_beta)
    n = brute.occupations(dets, sys.M)
    rng = np.random.default_rng(0)
    for d in rng.choice(len(n), 20, replace=False):
        e1, _, m1 = orc.local_energy(n[d], 0.0, direct=False)
        e2, _, m2 = orc.local_energy(n[d], 0.0, direct=True)
        assert len(m1) == len(m2)
        np.testing.assert_allclose(m1["ratio"], m2["ratio"], rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(e1, e2, rtol=1e-12)


def test_table_ratios_with_a_tiny_leading_pivot():
    """|psi(m)/psi(n)| from the G table against numpy determinants when C_occ's leading element is
    1e-17 next to entries of order one: the inverse needs the row exchange of partial pivoting (a
    first-non-zero pivot keeps the 1e-17 and loses every digit of the inverse's first column)."""
    sys = _h4()
    M = sys.M
    Ca = np.array([[1e-17, 1.0], [1.0, 1.0], [0.3, 0.5], [0.7, -0.2]])
    Cb = np.array([[0.9, 0.1], [-0.2, 0.8], [0.4, 0.3], [0.1, -0.6]])
    prm = S.Params(np.zeros((2 * M, 2 * M)), Ca, Cb)
    orc = Oracle(sys, prm)
    n = np.zeros(2 * M, dtype=np.uint8)
    n[[0, 1, M + 0, M + 1]] = 1
    _, _, mv = orc.local_energy(n, 0.0)
    assert len(mv) > 0

    def dets(occ):
        a = sorted(p for p in occ if p < M)
        b = sorted(p - M for p in occ if p >= M)
        return np.linalg.det(Ca[a]) * np.linalg.det(Cb[b])

    occ0 = [0, 1, M, M + 1]
    d0 = dets(occ0)
    for m in mv:
        occ = set(occ0) - {int(m["i"])} | {int(m["a"])}
        if m["kind"] == 2:
            occ = occ - {int(m["j"])} | {int(m["b"])}
        assert abs(abs(m["ratio"]) - abs(dets(occ) / d0)) <= 1e-12 * max(1.0, abs(dets(occ) / d0))


# --- in-place replacement convention and the a <-> b identity (Sec. III.B, Eq. R) -------
def test_double_contribution_is_inplace_minor_and_symmetric_in_ab():
    # The oracle's H_nm (explicit canonical phase) times psi(m)/psi(n) equals, for every double,
    # the in-place form <ab||ij> x (2x2 minor of G = C C_occ^-1) x Jastrow ratio with no sign
    # bookkeeping, and that form is unchanged when a and b are swapped (both factors flip sign).
    sys = _h6()
    prm = S.make_params(sys, seed=21, j_scale=0.1, c_noise=0.2)
    orc = Oracle(sys, prm)
    M, e = sys.M, sys.eri
    dets = brute.all_dets(sys.M, sys.n_alpha, sys.n_beta)
    n_all = brute.occupations(dets, sys.M)
    Jm = np.triu(prm.J)

    def logj(n):
        x = n.astype(float)
        return x @ Jm @ x                   # upper triangle incl. diagonal: sum_{p<=q} J_pq n_p n_q

    rng = np.random.default_rng(3)
    checked = 0
    for d in rng.choice(len(n_all), 12, replace=False):
        n = n_all[d]
        _, _, moves = orc.local_energy(n, 0.0)
        G, col = [], []
        for sg, C in ((0, prm.C_alpha), (1, prm.C_beta)):
            occ = np.flatnonzero(n[sg * M:(sg + 1) * M])
            G.append(C @ np.linalg.inv(C[occ]))
            col.append({int(k): c for c, k in enumerate(occ)})
        for mv in moves[moves["kind"] == 2]:
            i, j, a, b = (int(mv[f]) for f in ("i", "j", "a", "b"))
            si, sj = i // M, j // M
            pi, pj, pa, pb = i % M, j % M, a % M, b % M
            m = n.copy(); m[[i, j]] = 0; m[[a, b]] = 1
            jr = math.exp(logj(m) - logj(n))

            def inplace(pa, pb):
                if si == sj:
                    g, c = G[si], col[si]
                    v = e[pa, pi, pb, pj] - e[pa, pj, pb, pi]
                    minor = g[pa, c[pi]] * g[pb, c[pj]] - g[pa, c[pj]] * g[pb, c[pi]]
                else:
                    v = e[pa, pi, pb, pj]
                    minor = G[0][pa, col[0][pi]] * G[1][pb, col[1][pj]]
                return v * minor * jr

            ref = mv["h"] * mv["ratio"]
            got = inplace(pa, pb)
            assert abs(got - ref) <= 1e-10 * max(1.0, abs(ref)), (i, j, a, b)
            if si == sj:
                assert abs(inplace(pb, pa) - got) <= 1e-12 * max(1.0, abs(got))
            checked += 1
    assert checked > 100


# --- energy expectation and the variational bound (Eq. vmc) ------------------------------
def test_energy_is_rho_weighted_mean_and_variational(hub10):
    sys, prm, dets, H, n, psi = hub10
    orc = Oracle(sys, prm)
    el, _, _ = orc.local_energy_batch(n, 0.0)
    rho = psi ** 2 / np.sum(psi ** 2)
    e_vmc = float(np.sum(rho * el))
    e_exact = float(psi @ (H @ psi) / (psi @ psi))
    assert abs(e_vmc - e_exact) < 1e-10
    e0 = sla.eigsh(H, k=1, which="SA")[0][0]
    assert e_vmc >= e0 - 1e-10


# --- zero-variance: U=0, exact plane waves, no Jastrow -> E_L = -4(1+sqrt 5) t ----------
def test_zero_variance_free_fermions_ring10():
    sys = S.hubbard(10, 1, t=1.0, U=0.0)
    prm = S.make_params(sys, zero_jastrow=True, exact_planewave=True)
    orc = Oracle(sys, prm)
    dets = brute.all_dets(sys.M, 5, 5)
    n = brute.occupations(dets, sys.M)
    psi = brute.psi_all(n, sys.M, prm)
    keep = np.abs(psi) > 1e-8 * np.abs(psi).max()
    rng = np.random.default_rng(1)
    pick = rng.choice(np.nonzero(keep)[0], 300, replace=False)
    el, _, _ = orc.local_energy_batch(n[pick], 0.0)
    exact = -4.0 * (1.0 + math.sqrt(5.0))
    np.testing.assert_allclose(el, exact, rtol=0, atol=1e-9)


# --- screening: the kept set is exactly {S_ia > eps} U {|<ab||ij>| > eps} ----------------
@pytest.mark.parametrize("eps", [1e-3, 1e-2, 5e-2])
def test_screened_eloc_matches_filtered_brute(eps):
    sys = _h6()
    prm = S.make_params(sys, seed=3, j_scale=0.05, c_noise=0.1)
    dets, H = brute.hamiltonian(sys)
    n = brute.occupations(dets, sys.M)
    psi = brute.psi_all(n, sys.M, prm)
    Sia = brute.singles_bound(sys)
    M = sys.M
    orc = Oracle(sys, prm)
    Hc = H.tocoo()
    el_ref = np.zeros(len(dets))
    for r, c, v in zip(Hc.row, Hc.col, Hc.data):
        if r == c:
            el_ref[r] += v
            continue
        diff = dets[r] ^ dets[c]
        nbits = int(np.bitwise_count(diff))
        if nbits == 2:     # single: keep iff S_ia > eps
            p, q = [k for k in range(2 * M) if (int(diff) >> k) & 1]
            keep = Sia[p % M, q % M] > eps
        else:              # double: |H_nm| = |<ab||ij>|
            keep = abs(v) > eps
        if keep:
            el_ref[r] += v * psi[c] / psi[r]
    el, _, _ = orc.local_energy_batch(n, eps)
    np.testing.assert_allclose(el, el_ref, rtol=1e-10, atol=1e-10)


def test_eps_to_zero_limit():
    sys = _h6()
    prm = S.make_params(sys, seed=3)
    orc = Oracle(sys, prm)
    n = brute.occupations(brute.all_dets(sys.M, 3, 3), sys.M)[::37]
    e0, _, _ = orc.local_energy_batch(n, 0.0)
    errs = [np.max(np.abs(orc.local_energy_batch(n, eps)[0] - e0)) for eps in (1e-2, 1e-4, 1e-6, 1e-9)]
    assert errs[-1] < 1e-7 and errs[0] >= errs[1] >= errs[2] >= errs[3]


# --- CTMC: move-set symmetry (detailed balance, Sec. II.B) --------------------------------
def test_move_set_symmetric_and_detailed_balance():
    sys = _h6()
    prm = S.make_params(sys, seed=4, j_scale=0.05, c_noise=0.1)
    orc = Oracle(sys, prm)
    eps = 1e-3
    n_all = brute.occupations(brute.all_dets(sys.M, 3, 3), sys.M)
    rng = np.random.default_rng(2)
    for d in rng.choice(len(n_all), 15, replace=False):
        n = n_all[d]
        _, _, mv = orc.local_energy(n, eps)
        psin = orc.psi(n)
        for k in rng.choice(len(mv), min(10, len(mv)), replace=False):
            m = n.copy()
            o = mv[k]
            m[o["i"]] = 0
            m[o["a"]] = 1
            if o["kind"] == 2:
                m[o["j"]] = 0
                m[o["b"]] = 1
            _, _, back = orc.local_energy(m, eps)
            # the reverse move exists in m's screened set
            if o["kind"] == 1:
                sel = (back["kind"] == 1) & (back["i"] == o["a"]) & (back["a"] == o["i"])
            else:
                src = sorted([o["a"], o["b"]])
                dst = sorted([o["i"], o["j"]])
                sel = (back["kind"] == 2) & (back["i"] == src[0]) & (back["j"] == src[1]) \
                    & (back["a"] == dst[0]) & (back["b"] == dst[1])
            assert sel.sum() == 1
            r_fwd = abs(o["ratio"])
            r_bwd = abs(back[sel][0]["ratio"])
            psim = orc.psi(m)
            assert abs(psin ** 2 * r_fwd - psim ** 2 * r_bwd) <= 1e-10 * psin ** 2 * r_fwd


# --- Philox4x64-10 equals numpy's Philox bit generator (numpy pre-increments) -----------
@pytest.mark.parametrize("key,ctr", [((0, 0), (0, 0, 0, 0)), ((5, 7), (3, 0, 0, 0)),
                                     ((1807, 123456), (99, 1, 2, 3)),
                                     ((2 ** 64 - 1, 2 ** 63), (2 ** 64 - 2, 0, 0, 0))])
def test_philox_matches_numpy(key, ctr):
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(ctr, dtype=np.uint64))
    ref = bg.random_raw(4)
    c = list(ctr)
    c[0] = (c[0] + 1) % 2 ** 64
    np.testing.assert_array_equal(oracle.philox4x64(c, key), ref)


# --- CTMC choice frequencies follow r, residence time is 1/sum r (Sec. II.B) ------------
def test_ctmc_choice_distribution():
    rates = np.array([0.5, 1e-3, 2.0, 0.25, 0.0, 1.25])
    mv = np.zeros(rates.size, dtype=oracle.MOVE_DTYPE)
    mv["kind"] = 1
    mv["ratio"] = rates * np.array([1, -1, 1, -1, 1, 1])
    counts = np.zeros(rates.size)
    N = 40000
    t_ref = 1.0 / rates.sum()
    for step in range(N):
        rc, k, t = oracle.ctmc_choose(mv, seed=77, walker=3, step=step)
        assert rc == 0
        counts[k] += 1
        assert abs(t - t_ref) < 1e-14 * t_ref
    assert counts[4] == 0
    p = rates / rates.sum()
    chi2 = np.sum((counts - N * p)[p > 0] ** 2 / (N * p[p > 0]))
    assert chi2 < 25.0   # 4 degrees of freedom, p < 1e-4


# --- the choice rule at its boundaries, by exact integer arithmetic (reading 6 of Sec. II.B) ---
def _moves(ratios):
    mv = np.zeros(len(ratios), dtype=oracle.MOVE_DTYPE)
    mv["kind"] = 1
    mv["ratio"] = ratios
    return mv


def test_ctmc_choice_rule_at_exact_boundaries():
    """q_k = floor(r_k 2^64), Q = sum q_k, T = floor(U Q / 2^64), and the first move whose prefix
    sum exceeds T (strictly).  Two rates of 1/4 give q = 2^62 each and T = floor(U / 2): U = 2^63
    puts T exactly on the first prefix (move 1 is chosen), U = 2^63 - 1 just below it (move 0).
    Rates 1 and 2 give Q = 3 2^64 and T = 3U, so the first prefix 2^64 is crossed between
    U = floor((2^64 - 1) / 3) and the next U; U = 0 and U = 2^64 - 1 choose the first and the last
    move with a non-zero rate."""
    quarter = _moves([0.25, -0.25])
    assert oracle.ctmc_choose_u(quarter, 2 ** 63)[:2] == (0, 1)
    assert oracle.ctmc_choose_u(quarter, 2 ** 63 - 1)[:2] == (0, 0)
    rc, k, t = oracle.ctmc_choose_u(quarter, 0)
    assert (rc, k) == (0, 0) and t == 2.0
    big = _moves([1.0, 0.0, -2.0])
    u = (2 ** 64 - 1) // 3
    assert oracle.ctmc_choose_u(big, u)[:2] == (0, 0)
    assert oracle.ctmc_choose_u(big, u + 1)[:2] == (0, 2)
    assert oracle.ctmc_choose_u(big, 2 ** 64 - 1)[:2] == (0, 2)
    assert oracle.ctmc_choose_u(big, 0)[2] == 1.0 / 3.0
    # a rate below 2^-64 has q = 0 and is never chosen; no non-zero rate at all is reported
    tiny = _moves([0.0, 2.0 ** -70, 0.5])
    assert oracle.ctmc_choose_u(tiny, 0)[:2] == (0, 2)
    assert oracle.ctmc_choose_u(_moves([0.0, 2.0 ** -70]), 5)[0] == 1
    # the Philox form draws U as word 0 of Philox4x64-10(key = (seed, walker), counter = (step, 0, 0, 0))
    for step in range(5):
        U = int(oracle.philox4x64([step, 0, 0, 0], [77, 3])[0])
        assert oracle.ctmc_choose(big, seed=77, walker=3, step=step) == oracle.ctmc_choose_u(big, U)


# --- long-run CTMC: the time-weighted histogram converges to rho = psi^2 (Sec. II.B) ----
def test_ctmc_time_weighted_histogram_converges_to_rho():
    sys = _h4()
    prm = S.make_params(sys, seed=21, j_scale=0.1, c_noise=0.2)
    dets, _ = brute.hamiltonian(sys)
    nall = brute.occupations(dets, sys.M)
    psi = brute.psi_all(nall, sys.M, prm)
    rho = psi ** 2 / np.sum(psi ** 2)
    orc = Oracle(sys, prm)
    W, steps = 64, 1500
    rng = np.random.default_rng(3)
    n = np.ascontiguousarray(nall[rng.choice(len(nall), W)])
    ctr = np.zeros(W, dtype=np.uint64)
    hist = np.zeros(len(dets))
    weights = np.arange(2 * sys.M, dtype=np.uint64)
    for s in range(steps):
        masks = (n.astype(np.uint64) << weights[None, :]).sum(axis=1).astype(np.uint64)
        idx = np.searchsorted(dets, masks)
        _, tr, _, err = orc.sweep(n, 0.0, 1234, ctr)
        assert err == 0
        if s >= 100:
            np.add.at(hist, idx, tr)
    hist /= hist.sum()
    tv = 0.5 * np.abs(hist - rho).sum()
    assert tv < 0.03


# --- gradient ratios vs central finite differences of ln|psi| (Sec. III.B) --------------
def test_grad_logpsi_matches_finite_differences():
    sys = _h6()
    prm = S.make_params(sys, seed=8, j_scale=0.1, c_noise=0.2)
    orc = Oracle(sys, prm)
    M = sys.M
    n = brute.occupations(brute.all_dets(M, 3, 3), M)[123]
    dJ = np.zeros_like(prm.J)
    dCa = np.zeros_like(prm.C_alpha)
    dCb = np.zeros_like(prm.C_beta)
    orc.grad_logpsi(n, 1.0, dJ, dCa, dCb)

    def lnpsi(p):
        return math.log(abs(brute.psi_all(n[None], M, p)[0]))

    h = 1e-6
    rng = np.random.default_rng(4)
    for _ in range(12):
        p, q = sorted(rng.integers(0, 2 * M, 2))
        P1 = S.Params(prm.J.copy(), prm.C_alpha, prm.C_beta)
        P2 = S.Params(prm.J.copy(), prm.C_alpha, prm.C_beta)
        P1.J[p, q] += h
        P2.J[p, q] -= h
        fd = (lnpsi(P1) - lnpsi(P2)) / (2 * h)
        assert abs(fd - dJ[p, q]) < 1e-7
    for sg, (C, dC) in enumerate(((prm.C_alpha, dCa), (prm.C_beta, dCb))):
        for k in range(M):
            for x in range(C.shape[1]):
                Cp, Cm = C.copy(), C.copy()
                Cp[k, x] += h
                Cm[k, x] -= h
                if sg == 0:
                    P1, P2 = S.Params(prm.J, Cp, prm.C_beta), S.Params(prm.J, Cm, prm.C_beta)
                else:
                    P1, P2 = S.Params(prm.J, prm.C_alpha, Cp), S.Params(prm.J, prm.C_alpha, Cm)
                fd = (lnpsi(P1) - lnpsi(P2)) / (2 * h)
                assert abs(fd - dC[k, x]) < 1e-6 * max(1.0, abs(fd))


# --- energy gradient 2<(E_L - E) O>_rho equals dE/dp of the exact energy (Eq. grad) -----
def test_energy_gradient_matches_exact_derivative():
    sys = _h4()
    prm = S.make_params(sys, seed=12, j_scale=0.1, c_noise=0.2)
    dets, H = brute.hamiltonian(sys)
    M = sys.M
    n = brute.occupations(dets, M)
    orc = Oracle(sys, prm)

    def energy(p):
        psi = brute.psi_all(n, M, p)
        return float(psi @ (H @ psi) / (psi @ psi))

    psi = brute.psi_all(n, M, prm)
    rho = psi ** 2 / np.sum(psi ** 2)
    el, _, _ = orc.local_energy_batch(n, 0.0)
    E = float(np.sum(rho * el))
    dJ = np.zeros_like(prm.J)
    dCa = np.zeros_like(prm.C_alpha)
    dCb = np.zeros_like(prm.C_beta)
    for d in range(len(n)):
        orc.grad_logpsi(n[d], 2.0 * rho[d] * (el[d] - E), dJ, dCa, dCb)
    h = 1e-5
    for (p, q) in [(0, 1), (2, 5), (3, 3), (1, 6)]:
        P1 = S.Params(prm.J.copy(), prm.C_alpha, prm.C_beta)
        P2 = S.Params(prm.J.copy(), prm.C_alpha, prm.C_beta)
        P1.J[p, q] += h
        P2.J[p, q] -= h
        fd = (energy(P1) - energy(P2)) / (2 * h)
        assert abs(fd - dJ[p, q]) < 1e-7
    for (k, x) in [(0, 0), (3, 1), (2, 1)]:
        Cp, Cm = prm.C_alpha.copy(), prm.C_alpha.copy()
        Cp[k, x] += h
        Cm[k, x] -= h
        fd = (energy(S.Params(prm.J, Cp, prm.C_beta)) - energy(S.Params(prm.J, Cm, prm.C_beta))) / (2 * h)
        assert abs(fd - dCa[k, x]) < 1e-7


# --- AMSGrad recurrence, Eqs. (m1)-(m2) with the paper's defaults -----------------------
def test_amsgrad_hand_recurrence():
    alpha, b1, b2 = 0.01, 0.1, 0.01          # Sec. II.C defaults
    g_seq = [0.5, -1.0, 0.1]
    p = np.array([1.0]); m = np.zeros(1); v = np.zeros(1)
    # by hand:
    #   it1: m = 0.05,      v = max(0, 0.0025) = 0.0025,             p = 1 - 0.01*0.05/0.05 = 0.99
    #   it2: m = -0.055,    v = max(0.0025, 0.002475+0.01) = 0.012475, p = 0.99 + 0.01*0.055/sqrt(0.012475)
    #   it3: m = -0.0395,   v = max(0.012475, 0.01235025+0.0001) = 0.012475
    expect_p = [0.99, 0.99 + 0.01 * 0.055 / math.sqrt(0.012475),
                0.99 + 0.01 * 0.055 / math.sqrt(0.012475) + 0.01 * 0.0395 / math.sqrt(0.012475)]
    expect_v = [0.0025, 0.012475, 0.012475]
    for it, g in enumerate(g_seq):
        oracle.amsgrad(p, np.array([g]), m, v, alpha, b1, b2)
        assert abs(v[0] - expect_v[it]) < 1e-15
        assert abs(p[0] - expect_p[it]) < 1e-14
    # n = 0 gives no update
    p = np.array([2.0]); m = np.zeros(1); v = np.zeros(1)
    oracle.amsgrad(p, np.array([0.0]), m, v, alpha, b1, b2)
    assert p[0] == 2.0


def test_singles_screen_uses_two_electron_bound():
    """With the off-diagonal one-electron integrals removed, singles survive the screen only
    through the sum over j in S_ia (Sec. II.A); the filtered brute force must agree."""
    sys = _h6()
    sys.h1 = np.diag(np.diag(sys.h1)).copy()
    prm = S.make_params(sys, seed=3, j_scale=0.05, c_noise=0.1)
    dets, H = brute.hamiltonian(sys)
    n = brute.occupations(dets, sys.M)
    psi = brute.psi_all(n, sys.M, prm)
    Sia = brute.singles_bound(sys)
    vals = np.unique(np.round(Sia[~np.eye(sys.M, dtype=bool)], 12))
    mid = len(vals) // 2
    eps = float(0.5 * (vals[mid] + vals[mid + 1]))   # away from any S_ia (no near-ties)
    M = sys.M
    Hc = H.tocoo()
    el_ref = np.zeros(len(dets))
    n_single_kept = 0
    for r, c, v in zip(Hc.row, Hc.col, Hc.data):
        if r == c:
            el_ref[r] += v
            continue
        diff = int(dets[r] ^ dets[c])
        bits = [k for k in range(2 * M) if (diff >> k) & 1]
        keep = (Sia[bits[0] % M, bits[1] % M] > eps) if len(bits) == 2 else abs(v) > eps
        if keep:
            n_single_kept += len(bits) == 2
            el_ref[r] += v * psi[c] / psi[r]
    assert n_single_kept > 0
    el, _, _ = Oracle(sys, prm).local_energy_batch(n, eps)
    np.testing.assert_allclose(el, el_ref, rtol=1e-10, atol=1e-10)


def test_golden_constants_are_used_consistently():
    """The constants tests rely on match tests/golden/paper_values.json (each cited there)."""
    import json
    from pathlib import Path
    g = json.loads((Path(__file__).parent / "golden" / "paper_values.json").read_text())
    d = g["amsgrad_defaults"]
    assert (d["alpha"], d["beta1"], d["beta2"]) == (0.01, 0.1, 0.01)
    assert abs(g["free_fermion_ring10_energy"]["value"] + 4.0 * (1.0 + math.sqrt(5.0))) < 1e-12
