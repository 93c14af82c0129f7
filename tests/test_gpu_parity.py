"""GPU path against the oracle, element by element, through the C ABI (needs a GB300)."""
import numpy as np
import pytest
import torch

import oracle
from tests.gpu_common import make_case, oracle_n, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vmc():
    from paper_1807_10633_gb300 import vmc as v
    v.lib()
    return v


def _eloc_parity(vmc, name, W, eps, precision, tol, n_check=None, **pk):
    sys_, prm, occ = make_case(name, W, **pk)
    eng = vmc.Engine(sys_, prm, occ, eps=eps, precision=precision)
    e, t = eng.local_energy()
    eng.sync()
    e = e.cpu().numpy()
    t = t.cpu().numpy()
    idx = np.arange(W) if n_check is None else np.linspace(0, W - 1, n_check).astype(int)
    orc = oracle.Oracle(sys_, prm)
    ref, _, _ = orc.local_energy_batch(oracle_n(sys_, occ[idx]), eps)
    eng.close()
    return e[idx], ref, t[idx]


def test_eloc_fp64_hubbard10_all_walkers(vmc):
    e, ref, _ = _eloc_parity(vmc, "hubbard10", 256, 0.0, vmc.VMC_FP64, 1e-10)
    assert rel_err(e, ref) < 1e-10


def test_eloc_fp64_h20(vmc):
    e, ref, _ = _eloc_parity(vmc, "H20", 4096, 1e-6, vmc.VMC_FP64, 1e-10, n_check=512)
    assert rel_err(e, ref) < 1e-10


def test_eloc_mixed_h20(vmc):
    e, ref, _ = _eloc_parity(vmc, "H20", 1024, 1e-6, vmc.VMC_MIXED, 0, n_check=256)
    # 0.1 mEh per particle
    assert np.max(np.abs(e - ref)) < 1e-4 * 20


def _trajectory_parity(vmc, name, W, eps, steps, seed=4242):
    sys_, prm, occ = make_case(name, W)
    eng = vmc.Engine(sys_, prm, occ, eps=eps, precision=vmc.VMC_FP64)
    orc = oracle.Oracle(sys_, prm)
    n = np.ascontiguousarray(oracle_n(sys_, occ))
    ctr = np.zeros(W, dtype=np.uint64)
    for s in range(steps):
        e, t = eng.local_energy()
        codes = eng.ctmc_step(seed)
        el_ref, tr_ref, mv_ref, err = orc.sweep(n, eps, seed, ctr)
        assert err == 0
        assert rel_err(e.cpu().numpy(), el_ref) < 1e-10, f"step {s}"
        assert rel_err(t.cpu().numpy(), tr_ref) < 1e-12, f"step {s}"
        mv = vmc.decode_moves(codes.cpu().numpy())
        np.testing.assert_array_equal(mv, mv_ref.astype(np.int64), err_msg=f"step {s}")
        np.testing.assert_array_equal(eng.occupations(), n, err_msg=f"step {s}")
    eng.sync()
    eng.close()


def test_ctmc_trajectory_hubbard10_2000_steps(vmc):
    _trajectory_parity(vmc, "hubbard10", 256, 0.0, 2000)


def test_ctmc_trajectory_h20(vmc):
    _trajectory_parity(vmc, "H20", 512, 1e-6, 30)
