"""Gradient ratios, AMSGrad, energy gradient and table updates on the GPU vs the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1807_10633_gb300 import systems as S
from tests.gpu_common import make_case, oracle_n, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vmc():
    from paper_1807_10633_gb300 import vmc as v
    v.lib()
    return v


@pytest.mark.parametrize("precision,tol", [(0, 1e-11), (1, 2e-5)])
def test_vjp_matches_oracle_sum(vmc, precision, tol):
    sys_, prm, occ = make_case("H20", 777)     # ragged walker count (not a multiple of a chunk)
    eng = vmc.Engine(sys_, prm, occ, eps=1e-6, precision=precision)
    rng = np.random.default_rng(5)
    w = rng.normal(size=eng.W)
    dJ, dCa, dCb = eng.grad_logpsi(torch.tensor(w, device="cuda"))
    eng.sync()
    orc = oracle.Oracle(sys_, prm)
    n = oracle_n(sys_, occ)
    rJ = np.zeros_like(prm.J); rA = np.zeros_like(prm.C_alpha); rB = np.zeros_like(prm.C_beta)
    for k in range(eng.W):
        orc.grad_logpsi(n[k], w[k], rJ, rA, rB)
    scale = np.abs(w).sum()
    assert np.max(np.abs(dJ.cpu().numpy() - rJ)) <= tol * scale
    assert np.max(np.abs(dCa.cpu().numpy() - rA)) <= tol * scale * max(1, np.abs(rA).max())
    assert np.max(np.abs(dCb.cpu().numpy() - rB)) <= tol * scale * max(1, np.abs(rB).max())
    eng.close()


@pytest.mark.parametrize("name,W", [("H6", 1), ("hubbard10", 33), ("H20", 777), ("H100", 2049), ("H160", 4099)])
def test_jastrow_sums_tensor_cores_equal_integer_pipe(vmc, name, W):
    """The tcgen05 digit-product path and the integer-pipe path give bit-identical Jastrow sums,
    for the VJP and for the accumulated (t, t E_L) pair: spin-orbital counts inside one tile and
    across several (ragged last tile), ragged walker counts, weights over nine decades."""
    sys_, prm, occ = make_case(name, W)
    eng = vmc.Engine(sys_, prm, occ, eps=1e-6, precision=vmc.VMC_MIXED)
    try:
        rng = np.random.default_rng(11)
        w = torch.tensor(rng.normal(size=W) * 10.0 ** rng.integers(-4, 5, size=W), device="cuda")
        t = torch.tensor(np.abs(rng.normal(size=W)) + 0.1, device="cuda")
        e = torch.tensor(rng.normal(size=W) * 50.0, device="cuda")
        res = []
        for tc in (1, 0):
            vmc.vmc_set_option(eng.ctx, vmc.VMC_OPT_GRAD_J_TENSOR_CORES, tc)
            dJ, _, _ = eng.grad_logpsi(w)
            AO = torch.zeros(eng.n_params, dtype=torch.float64, device="cuda")
            AEO = torch.zeros_like(AO)
            sums = torch.zeros(2, dtype=torch.float64, device="cuda")
            vmc.vmc_accumulate_gradient(eng.ctx, eng.walkers.struct(), t, e, eng.split(AO), eng.split(AEO), sums)
            eng.sync()
            res.append((dJ.cpu().numpy(), AO.cpu().numpy(), AEO.cpu().numpy()))
        for a, b in zip(*res):
            assert np.array_equal(a, b)
        assert np.abs(res[0][0]).max() > 0 and np.abs(res[0][2]).max() > 0
    finally:
        eng.close()


def test_amsgrad_matches_oracle(vmc):
    rng = np.random.default_rng(6)
    n = 100_003
    p0 = rng.normal(size=n); m0 = rng.normal(size=n) * 0.1; v0 = np.abs(rng.normal(size=n)) * 0.01
    v0[::7] = 0.0
    g = rng.normal(size=n)
    g[::11] = 0.0
    ctx = vmc.vmc_create(0, torch.cuda.current_stream())
    P = torch.tensor(p0, device="cuda"); Mt = torch.tensor(m0, device="cuda"); V = torch.tensor(v0, device="cuda")
    vmc.vmc_amsgrad_update(ctx, P, torch.tensor(g, device="cuda"), Mt, V, 0.01, 0.1, 0.01)
    vmc.vmc_sync(ctx)
    p1, m1, v1 = p0.copy(), m0.copy(), v0.copy()
    oracle.amsgrad(p1, g, m1, v1, 0.01, 0.1, 0.01)
    assert rel_err(P.cpu().numpy(), p1) < 1e-14
    assert rel_err(Mt.cpu().numpy(), m1) < 1e-14
    assert rel_err(V.cpu().numpy(), v1) < 1e-14
    vmc.vmc_destroy(ctx)


def test_energy_gradient_and_walker_reduce(vmc):
    rng = np.random.default_rng(7)
    W, n = 1000, 5000
    t = rng.random(W); e = rng.normal(size=W) - 5
    aO = rng.normal(size=n); aEO = rng.normal(size=n)
    ctx = vmc.vmc_create(0, torch.cuda.current_stream())
    sums = torch.zeros(2, dtype=torch.float64, device="cuda")
    vmc.vmc_walker_reduce(ctx, W, torch.tensor(t, device="cuda"), torch.tensor(e, device="cuda"), sums)
    g = torch.zeros(n, dtype=torch.float64, device="cuda")
    vmc.vmc_energy_gradient(ctx, sums, torch.tensor(aO, device="cuda"), torch.tensor(aEO, device="cuda"), g)
    vmc.vmc_sync(ctx)
    T = t.sum(); E = (t * e).sum() / T
    assert abs(sums[0].item() - T) < 1e-12 * T and abs(sums[1].item() - (t * e).sum()) < 1e-11 * abs((t * e).sum())
    assert rel_err(g.cpu().numpy(), 2 * (aEO / T - E * aO / T)) < 1e-12
    vmc.vmc_destroy(ctx)


def test_log_psi_matches_oracle_and_autograd_matches_finite_differences(vmc):
    sys_, prm, occ = make_case("H6", 40, j_scale=0.1, c_noise=0.2)
    eng = vmc.Engine(sys_, prm, occ, eps=1e-8, precision=vmc.VMC_FP64)
    lp = eng.log_psi().cpu().numpy()
    orc = oracle.Oracle(sys_, prm)
    n = oracle_n(sys_, occ)
    ref = np.array([np.log(abs(orc.psi(n[k]))) for k in range(eng.W)])
    assert rel_err(lp, ref) < 1e-12
    J = eng.J.clone().requires_grad_(True)
    Ca = eng.Ca.clone().requires_grad_(True)
    Cb = eng.Cb.clone().requires_grad_(True)
    wts = torch.randn(eng.W, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    out = vmc.LogPsi.apply(J, Ca, Cb, eng)
    (out * wts).sum().backward()
    h = 1e-6
    rng = np.random.default_rng(8)

    def f(Jx, Cax, Cbx):
        o = torch.zeros(eng.W, dtype=torch.float64, device="cuda")
        vmc.vmc_log_psi(eng.ctx, eng.walkers.struct(), vmc.params_struct(Jx, Cax, Cbx), o)
        return float((o * wts).sum())

    for _ in range(8):
        p, q = sorted(rng.integers(0, 2 * sys_.M, 2))
        Jp = eng.J.clone(); Jp[p, q] += h
        Jm = eng.J.clone(); Jm[p, q] -= h
        fd = (f(Jp, eng.Ca, eng.Cb) - f(Jm, eng.Ca, eng.Cb)) / (2 * h)
        assert abs(fd - J.grad[p, q].item()) < 1e-6 * max(1, abs(fd))
    for _ in range(8):
        k, x = rng.integers(0, sys_.M), rng.integers(0, sys_.n_alpha)
        Cp = eng.Ca.clone(); Cp[k, x] += h
        Cm = eng.Ca.clone(); Cm[k, x] -= h
        fd = (f(eng.J, Cp, eng.Cb) - f(eng.J, Cm, eng.Cb)) / (2 * h)
        assert abs(fd - Ca.grad[k, x].item()) < 1e-6 * max(1, abs(fd))
    eng.close()


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 2e-4)])
def test_sherman_morrison_tables_equal_recomputed(vmc, precision, tol):
    sys_, prm, occ = make_case("H20", 256)
    eng = vmc.Engine(sys_, prm, occ, eps=1e-6, precision=precision)
    for s in range(40):
        eng.local_energy()
        eng.ctmc_step(77)
    eng.sync()
    def g_by_orbital():
        # G rows are virtual slots; a full recompute renumbers the slots, so compare by orbital
        M, na, nb, W = sys_.M, sys_.n_alpha, sys_.n_beta, eng.W
        G = eng.walkers.G.double().cpu().numpy().reshape(W, -1)
        V = eng.walkers.virt_list.cpu().numpy().astype(np.int64).reshape(W, -1)
        out = np.zeros((W, 2, M, max(na, nb)))
        for w in range(W):
            ga = G[w, :(M - na) * na].reshape(M - na, na)
            gb = G[w, (M - na) * na:].reshape(M - nb, nb)
            out[w, 0, V[w, :M - na], :na] = ga
            out[w, 1, V[w, M - na:], :nb] = gb
        return out

    G1 = g_by_orbital()
    A1, S1, F1, E1 = (x.clone() for x in (eng.walkers.AinvT, eng.walkers.S, eng.walkers.F, eng.walkers.e_diag))
    eng.init()      # full recompute from the (moved) occupations, same column order
    eng.sync()
    G2 = g_by_orbital()
    assert np.max(np.abs(G1 - G2)) <= tol * max(1.0, np.abs(G2).max())
    for a, b in [(A1, eng.walkers.AinvT), (S1, eng.walkers.S)]:
        a = a.double().cpu().numpy(); b = b.double().cpu().numpy()
        assert np.max(np.abs(a - b)) <= tol * max(1.0, np.abs(b).max())
    # F: FP64 updates are exact sums of table values; FP32 ones round at every move
    f1, f2 = F1.double().cpu().numpy(), eng.walkers.F.double().cpu().numpy()
    assert np.max(np.abs(f1 - f2)) < (1e-11 if precision == 0 else 2e-5 * max(1.0, np.abs(f2).max()))
    assert np.max(np.abs(E1.cpu().numpy() - eng.walkers.e_diag.cpu().numpy())) < 1e-10
    eng.close()


def test_logpsi_refuses_parameters_other_than_the_tables(vmc):
    """The backward uses the walker tables, so a call with other parameter values (a perturbed copy,
    or the engine's own parameters changed in place without a refresh) must raise; after the values
    are copied in and the tables refreshed, the gradient matches central differences."""
    sys_, prm, occ = make_case("H6", 32)
    eng = vmc.Engine(sys_, prm, occ, eps=1e-6, precision=0)
    Ca = (eng.Ca + 1e-3).clone().requires_grad_(True)
    with pytest.raises(ValueError, match="refresh"):
        vmc.LogPsi.apply(eng.J.clone(), Ca, eng.Cb.clone(), eng)
    eng.Ca.add_(1e-3)                                   # parameters moved, tables not refreshed
    with pytest.raises(ValueError, match="refresh"):
        vmc.LogPsi.apply(eng.J.clone(), Ca, eng.Cb.clone(), eng)
    eng.refresh()
    out = vmc.LogPsi.apply(eng.J.clone(), Ca, eng.Cb.clone(), eng)
    wts = torch.linspace(-1.0, 1.0, eng.W, dtype=torch.float64, device="cuda")
    (out * wts).sum().backward()
    h = 1e-6

    def f(Cax):
        o = torch.zeros(eng.W, dtype=torch.float64, device="cuda")
        vmc.vmc_log_psi(eng.ctx, eng.walkers.struct(), vmc.params_struct(eng.J, Cax, eng.Cb), o)
        return float((o * wts).sum())

    for k, x in ((0, 0), (2, 1), (5, 2)):
        Cp = eng.Ca.clone(); Cp[k, x] += h
        Cm = eng.Ca.clone(); Cm[k, x] -= h
        fd = (f(Cp) - f(Cm)) / (2 * h)
        assert abs(fd - Ca.grad[k, x].item()) < 1e-6 * max(1, abs(fd))
    eng.close()
