"""Full-size parity: the H160 chain (STO-3G, 1.8 bohr, Loewdin orbitals, 80 alpha + 80 beta),
eps = 1e-6, 32,768 walkers, the inputs and the launch configuration the benchmark times (same seeds,
autotuned local-energy CTA width).  The oracle recomputes sampled walkers one by one: E_L and the
residence time (Sec. II.A-B), the CTMC choice with the walker's own Philox key (FP64 form), and the
gradient vector-Jacobian product with weights on the sampled walkers only (Sec. III.B)."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_1807_10633_gb300 import systems as S
from tests.gpu_common import oracle_n, rel_err

pytestmark = pytest.mark.gpu

W = 32768
EPS = 1e-6
SEED = 4242
SAMPLE = np.linspace(0, W - 1, 12).astype(int)


@pytest.fixture(scope="module")
def vmc():
    from paper_1807_10633_gb300 import vmc as v
    v.lib()
    return v


@pytest.fixture(scope="module")
def h160():
    sys_ = S.named_system("H160")
    prm = S.make_params(sys_, seed=S.MASTER_SEED)
    occ = S.init_occupations(sys_, prm, W, seed=S.MASTER_SEED + 1)
    orc = oracle.Oracle(sys_, prm)
    n = np.ascontiguousarray(oracle_n(sys_, occ[SAMPLE]))
    el, _, _ = orc.local_energy_batch(n, EPS, n_threads=os.cpu_count() or 1)
    return sys_, prm, occ, orc, n, el


# form: (precision, FP32 Gauss-Jordan refresh option)
FORMS = {"fp64": (0, 0), "mixed": (1, 0), "mixed_gj32": (1, 1)}


@pytest.mark.parametrize("form", list(FORMS))
def test_h160_full_size(vmc, h160, form):
    sys_, prm, occ, orc, n, el_ref = h160
    precision, gj32 = FORMS[form]
    eng = vmc.Engine(sys_, prm, occ, eps=EPS, precision=precision)
    try:
        if gj32:
            vmc.vmc_set_option(eng.ctx, vmc.VMC_OPT_MIXED_REFRESH_GJ32, 1)
            eng.refresh()
        threads = vmc.Batch([eng]).autotune()
        assert threads in (128, 256, 384, 512)
        e, t = eng.local_energy()
        codes = eng.ctmc_step(SEED)
        eng.sync()
        e = e.cpu().numpy()[SAMPLE]
        t = t.cpu().numpy()[SAMPLE]
        if precision == 0:
            assert rel_err(e, el_ref) < 1e-10
        else:
            err = np.max(np.abs(e - el_ref)) / sys_.n_elec
            print(f"H160 {form}: max |dE_L| per electron {1e3 * err:.3e} mEh")
            assert err < 1e-4                                   # 0.1 mEh per particle
        # residence time and the CTMC choice of each sampled walker (counter 0, key (seed, walker))
        mv = vmc.decode_moves(codes.cpu().numpy()[SAMPLE])
        for r, w in enumerate(SAMPLE):
            _, _, moves = orc.local_energy(n[r], EPS)
            rc, k, tr = oracle.ctmc_choose(moves, SEED, int(w), 0)
            assert rc == 0 and k >= 0
            if precision == 0:
                assert abs(t[r] - tr) <= 1e-12 * tr
                ref = moves[k]
                assert tuple(mv[r]) == (ref["kind"], ref["i"], ref["j"], ref["a"], ref["b"]), f"walker {w}"
            else:
                assert abs(t[r] - tr) <= 1e-4 * tr
        # gradient VJP with weights on the sampled walkers only (the state before the move)
        eng2 = vmc.Engine(sys_, prm, occ, eps=EPS, precision=precision)
        try:
            if gj32:
                vmc.vmc_set_option(eng2.ctx, vmc.VMC_OPT_MIXED_REFRESH_GJ32, 1)
                eng2.refresh()
            rng = np.random.default_rng(17)
            wv = np.zeros(W)
            wv[SAMPLE] = rng.normal(size=SAMPLE.size)
            dJ, dCa, dCb = eng2.grad_logpsi(torch.tensor(wv, device="cuda"))
            eng2.sync()
        finally:
            eng2.close()
        rJ = np.zeros_like(prm.J); rA = np.zeros_like(prm.C_alpha); rB = np.zeros_like(prm.C_beta)
        for r, w in enumerate(SAMPLE):
            orc.grad_logpsi(n[r], wv[w], rJ, rA, rB)
        scale = np.abs(wv).sum()
        tol = 1e-11 if precision == 0 else 2e-5
        assert np.max(np.abs(dJ.cpu().numpy() - rJ)) <= tol * scale
        assert np.max(np.abs(dCa.cpu().numpy() - rA)) <= tol * scale * max(1, np.abs(rA).max())
        assert np.max(np.abs(dCb.cpu().numpy() - rB)) <= tol * scale * max(1, np.abs(rB).max())
    finally:
        eng.close()
