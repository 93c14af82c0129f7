"""The correlator-product wavefunction of Sec. III.A on the GPU against the oracle (needs a GB300).

psi(n) = prod_l c_l[n_l] x pair Jastrow x det C^a det C^b with local 5-site correlators (clipped
windows on a chain, periodic on a ring, site + 4 neighbours on a lattice).  Through the C ABI:
FP64 local energies within 1e-10 relative, CTMC trajectories bit-exact in moves and occupations,
the screened move set with its rates, ln|psi|, the gradient ratios d ln psi / dc = 1/c summed over
walkers (vector-Jacobian product within 1e-11 sum|w|), the energy-gradient pieces, and the mixed
form within 0.1 mEh per electron.  The pair Jastrow rewritten as one- and two-site correlators must
reproduce the pair-Jastrow kernels."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1807_10633_gb300 import systems as S
from tests.gpu_common import oracle_n, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vmc():
    from paper_1807_10633_gb300 import vmc as v
    v.lib()
    return v


def _case(name, W, seed=S.MASTER_SEED, noise=0.1, j_scale=0.01):
    sys_ = S.named_system(name)
    prm = S.make_params(sys_, seed=seed, j_scale=j_scale, c_noise=0.05)
    cps = S.make_cps(sys_, seed=seed + 7, noise=noise)
    occ = S.init_occupations(sys_, prm, W, seed=seed + 1)
    return sys_, prm, cps, occ


@pytest.mark.parametrize("name,W,eps,n_check", [("hubbard10", 256, 0.0, 256), ("hubbard4x4", 256, 0.0, 64),
                                                ("H20", 1024, 1e-6, 128), ("H40", 512, 1e-6, 32)])
def test_cps_local_energy_fp64(vmc, name, W, eps, n_check):
    sys_, prm, cps, occ = _case(name, W)
    eng = vmc.Engine(sys_, prm, occ, eps=eps, precision=vmc.VMC_FP64, cps=cps)
    try:
        e, t = eng.local_energy()
        eng.sync()
        idx = np.linspace(0, W - 1, n_check).astype(int)
        el_ref, _, _ = oracle.Oracle(sys_, prm, cps).local_energy_batch(oracle_n(sys_, occ[idx]), eps)
        assert rel_err(e.cpu().numpy()[idx], el_ref) < 1e-10
        lp = eng.log_psi().cpu().numpy()[idx]
        orc = oracle.Oracle(sys_, prm, cps)
        ref = np.array([math.log(abs(orc.psi(x))) for x in oracle_n(sys_, occ[idx[:16]])])
        assert rel_err(lp[:16], ref) < 1e-12
    finally:
        eng.close()


def test_cps_local_energy_mixed(vmc):
    sys_, prm, cps, occ = _case("H20", 1024)
    eng = vmc.Engine(sys_, prm, occ, eps=1e-6, precision=vmc.VMC_MIXED, cps=cps)
    try:
        e, _ = eng.local_energy()
        eng.sync()
        idx = np.arange(0, 1024, 8)
        el_ref, _, _ = oracle.Oracle(sys_, prm, cps).local_energy_batch(oracle_n(sys_, occ[idx]), 1e-6)
        assert np.max(np.abs(e.cpu().numpy()[idx] - el_ref)) < 1e-4 * sys_.n_elec
    finally:
        eng.close()


@pytest.mark.parametrize("name,W,eps,steps", [("hubbard10", 256, 0.0, 300), ("H20", 256, 1e-6, 30)])
def test_cps_ctmc_trajectory_bit_exact(vmc, name, W, eps, steps):
    sys_, prm, cps, occ = _case(name, W)
    eng = vmc.Engine(sys_, prm, occ, eps=eps, precision=vmc.VMC_FP64, cps=cps)
    orc = oracle.Oracle(sys_, prm, cps)
    n = np.ascontiguousarray(oracle_n(sys_, occ))
    ctr = np.zeros(W, dtype=np.uint64)
    seed = 777
    try:
        for s in range(steps):
            e, t = eng.local_energy()
            codes = eng.ctmc_step(seed)
            el_ref, tr_ref, mv_ref, err = orc.sweep(n, eps, seed, ctr)
            assert err == 0
            assert rel_err(e.cpu().numpy(), el_ref) < 1e-10, f"step {s}"
            assert rel_err(t.cpu().numpy(), tr_ref) < 1e-12, f"step {s}"
            np.testing.assert_array_equal(vmc.decode_moves(codes.cpu().numpy()), mv_ref.astype(np.int64),
                                          err_msg=f"step {s}")
            np.testing.assert_array_equal(eng.occupations(), n, err_msg=f"step {s}")
        eng.sync()
        # the correlator indices kept up to date by the moves equal indices rebuilt from scratch
        kept = eng.walkers.cps_state.clone()
        eng.refresh()
        eng.sync()
        assert torch.equal(kept, eng.walkers.cps_state)
    finally:
        eng.close()


def test_cps_screened_moves_match_the_oracle(vmc):
    sys_, prm, cps, occ = _case("H20", 64)
    eng = vmc.Engine(sys_, prm, occ, eps=1e-6, precision=vmc.VMC_FP64, cps=cps)
    orc = oracle.Oracle(sys_, prm, cps)
    try:
        per, cnt, _ = eng.screened_moves(0, 16)
        for w in range(16):
            _, _, mv = orc.local_energy(oracle_n(sys_, occ[w:w + 1])[0], 1e-6)
            code, ratio, contrib = per[w]
            want = np.stack([mv["kind"], mv["i"], mv["j"], mv["a"], mv["b"]], axis=1).astype(np.int64)
            np.testing.assert_array_equal(vmc.decode_moves(code), want)
            r_ref = np.abs(mv["ratio"])
            assert np.all(np.abs(np.abs(ratio) - r_ref) <= 1e-10 * (r_ref + 1e-3 * r_ref.max()))
    finally:
        eng.close()


@pytest.mark.parametrize("precision,tol", [(0, 1e-11), (1, 1e-6)])
def test_cps_gradient_vjp_and_accumulation(vmc, precision, tol):
    sys_, prm, cps, occ = _case("H20", 2048)
    eng = vmc.Engine(sys_, prm, occ, eps=1e-6, precision=precision, cps=cps)
    orc = oracle.Oracle(sys_, prm, cps)
    n = oracle_n(sys_, occ)
    rng = np.random.default_rng(5)
    try:
        w = torch.tensor(rng.normal(size=eng.W), device="cuda")
        dc = eng.grad_logpsi_cps(w)
        ref = np.zeros(eng.n_cps)
        wn = w.cpu().numpy()
        for k in range(eng.W):
            orc.grad_cps(n[k], float(wn[k]), ref)
        scale = float(np.abs(wn).sum())
        assert np.max(np.abs(dc.cpu().numpy() - ref)) <= 1e-11 * scale * max(1.0, np.abs(ref).max())
        # energy-gradient pieces over one sweep: sum t O and sum t E_L O
        e, t = eng.local_energy()
        ao = torch.zeros_like(eng.c)
        aeo = torch.zeros_like(eng.c)
        vmc.vmc_accumulate_gradient_cps(eng.ctx, eng.walkers.struct(), eng.params, t, e, ao, aeo)
        eng.sync()
        tn, en = t.cpu().numpy(), e.cpu().numpy()
        r_o, r_eo = np.zeros(eng.n_cps), np.zeros(eng.n_cps)
        for k in range(eng.W):
            orc.grad_cps(n[k], float(tn[k]), r_o)
            orc.grad_cps(n[k], float(tn[k] * en[k]), r_eo)
        assert np.max(np.abs(ao.cpu().numpy() - r_o)) <= tol * float(np.abs(tn).sum()) * max(1.0, np.abs(r_o).max())
        assert np.max(np.abs(aeo.cpu().numpy() - r_eo)) <= tol * float(np.abs(tn * en).sum()) * max(1.0, np.abs(r_eo).max())
    finally:
        eng.close()


def test_cps_gradient_is_deterministic(vmc):
    sys_, prm, cps, occ = _case("H20", 4096)
    eng = vmc.Engine(sys_, prm, occ, eps=1e-6, precision=vmc.VMC_MIXED, cps=cps)
    try:
        w = torch.linspace(-1.0, 2.0, eng.W, dtype=torch.float64, device="cuda")
        a = eng.grad_logpsi_cps(w)
        b = eng.grad_logpsi_cps(w)
        eng.sync()
        assert torch.equal(a, b)
    finally:
        eng.close()


def _jastrow_as_cps(J, M):
    """The pair Jastrow as one- and two-site correlators (site p: the alpha/beta terms of p; pair
    (p, q): the four cross terms), from the upper triangle of J."""
    sites, vals = [], []
    for p in range(M):
        a, b = p, M + p
        v = [math.exp(J[a, a] * (st & 1) + J[b, b] * (st >> 1) + J[a, b] * (st & 1) * (st >> 1)) for st in range(4)]
        sites.append(np.array([p], dtype=np.int32)); vals.append(np.array(v))
    for p in range(M):
        for q in range(p + 1, M):
            v = []
            for st in range(16):
                npa, npb, nqa, nqb = st & 1, (st >> 1) & 1, (st >> 2) & 1, (st >> 3) & 1
                v.append(math.exp(J[p, q] * npa * nqa + J[p, M + q] * npa * nqb + J[q, M + p] * npb * nqa
                                  + J[M + p, M + q] * npb * nqb))
            sites.append(np.array([p, q], dtype=np.int32)); vals.append(np.array(v))
    return S.CPS(sites, vals)


def test_pair_jastrow_as_correlators_reproduces_the_pair_kernels(vmc):
    sys_ = S.named_system("hubbard10")
    prm = S.make_params(sys_, seed=3, j_scale=0.05)
    occ = S.init_occupations(sys_, prm, 128, seed=4)
    ref = vmc.Engine(sys_, prm, occ, eps=0.0, precision=vmc.VMC_FP64)
    cps = _jastrow_as_cps(prm.J, sys_.M)
    prm0 = S.Params(np.zeros_like(prm.J), prm.C_alpha, prm.C_beta)
    got = vmc.Engine(sys_, prm0, occ, eps=0.0, precision=vmc.VMC_FP64, cps=cps)
    try:
        for s in range(20):
            e0, t0 = ref.local_energy()
            e1, t1 = got.local_energy()
            assert rel_err(e1.cpu().numpy(), e0.cpu().numpy()) < 1e-12, s
            assert rel_err(t1.cpu().numpy(), t0.cpu().numpy()) < 1e-12, s
            m0 = ref.ctmc_step(11)
            m1 = got.ctmc_step(11)
            assert torch.equal(m0, m1), s
    finally:
        ref.close()
        got.close()


def test_cps_h160_sampled_walkers(vmc):
    """The H160 chain with 5-site correlators (~1.6e5 coefficients): sampled walkers of the
    benchmark's walker count against the oracle, FP64 and mixed forms."""
    sys_, prm, cps, occ = _case("H160", 4096)
    idx = np.array([0, 1365, 2730, 4095])
    import os
    el_ref, _, _ = oracle.Oracle(sys_, prm, cps).local_energy_batch(oracle_n(sys_, occ[idx]), 1e-6,
                                                                    n_threads=os.cpu_count() or 1)
    for precision in (vmc.VMC_FP64, vmc.VMC_MIXED):
        eng = vmc.Engine(sys_, prm, occ, eps=1e-6, precision=precision, cps=cps)
        try:
            vmc.Batch([eng]).autotune()
            e, _ = eng.local_energy()
            eng.sync()
            e = e.cpu().numpy()[idx]
            if precision == vmc.VMC_FP64:
                assert rel_err(e, el_ref) < 1e-10
            else:
                assert np.max(np.abs(e - el_ref)) < 1e-4 * sys_.n_elec
        finally:
            eng.close()
