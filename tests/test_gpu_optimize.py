"""The optimisation loop (Sec. II.C) on the GPU against the same loop built from the oracle's
pieces: per iteration, the time-weighted energy of Eq. (vmc) and, after the AMSGrad step, every
parameter (FP64 form; CTMC choices bit-exact, so both loops visit the same determinants)."""
from types import SimpleNamespace

import numpy as np
import pytest

import oracle
from paper_1807_10633_gb300 import systems as S
from tests.gpu_common import make_case, oracle_n, rel_err

pytestmark = pytest.mark.gpu


def _split(p, M, na, nb):
    N2 = 2 * M
    a, b = N2 * N2, N2 * N2 + M * na
    return p[:a].reshape(N2, N2), p[a:b].reshape(M, na), p[b:b + M * nb].reshape(M, nb)


def _oracle_loop(sys_, prm, occ, n_iter, sweeps, seed, eps, alpha0, alpha1, warm):
    M, na, nb = sys_.M, sys_.n_alpha, sys_.n_beta
    p = prm.flat().astype(np.float64).copy()
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    n = np.ascontiguousarray(oracle_n(sys_, occ))
    ctr = np.zeros(occ.shape[0], dtype=np.uint64)
    energies, params = [], []
    for k in range(n_iter):
        J, Ca, Cb = _split(p, M, na, nb)
        orc = oracle.Oracle(sys_, SimpleNamespace(J=J.copy(), C_alpha=Ca.copy(), C_beta=Cb.copy()))
        AO = np.zeros_like(p)
        AEO = np.zeros_like(p)
        aoJ, aoA, aoB = (np.ascontiguousarray(x) for x in _split(AO, M, na, nb))
        aeJ, aeA, aeB = (np.ascontiguousarray(x) for x in _split(AEO, M, na, nb))
        T = TE = 0.0
        for _ in range(sweeps):
            before = n.copy()
            el, tr, _, err = orc.sweep(n, eps, seed + k, ctr)
            assert err == 0
            for w in range(n.shape[0]):
                orc.grad_logpsi(before[w], tr[w], aoJ, aoA, aoB)
                orc.grad_logpsi(before[w], tr[w] * el[w], aeJ, aeA, aeB)
            T += tr.sum()
            TE += (tr * el).sum()
        AO = np.concatenate([aoJ.ravel(), aoA.ravel(), aoB.ravel()])
        AEO = np.concatenate([aeJ.ravel(), aeA.ravel(), aeB.ravel()])
        g = 2.0 * (AEO / T - (TE / T) * (AO / T))                      # Eq. (grad)
        oracle.amsgrad(p, g, m, v, alpha0 if k < warm else alpha1, 0.1, 0.01)
        energies.append(TE / T)
        params.append(p.copy())
    return np.array(energies), params


@pytest.mark.parametrize("name,W,eps", [("H4", 96, 1e-8), ("hubbard6", 64, 0.0)])
def test_optimisation_loop_matches_oracle(name, W, eps):
    from paper_1807_10633_gb300 import optimize as O
    from paper_1807_10633_gb300 import vmc
    vmc.lib()
    n_iter, sweeps, seed = 7, 3, 99
    sys_, prm, occ = make_case(name, W, j_scale=0.05, c_noise=0.1)
    eng = vmc.Engine(sys_, prm, occ, eps=eps, precision=vmc.VMC_FP64)
    seen = []
    try:
        its = O.optimize(eng, n_iter, sweeps, seed=seed, warm=3,
                         callback=lambda it: seen.append(eng.p.cpu().numpy().copy()))
    finally:
        eng.close()
    ref_e, ref_p = _oracle_loop(sys_, prm, occ, n_iter, sweeps, seed, eps, 0.001, 0.01, 3)
    got_e = np.array([it.energy for it in its])
    assert rel_err(got_e, ref_e) < 1e-10
    for k in range(n_iter):
        assert np.max(np.abs(seen[k] - ref_p[k])) < 1e-10, f"iteration {k}"
    assert [it.alpha for it in its] == [0.001] * 3 + [0.01] * (n_iter - 3)

