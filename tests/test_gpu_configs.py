"""Parity at the full sizes of two more benchmark configurations, on walkers the oracle recomputes
one by one (mixed form: 0.1 mEh per electron):

- the H80 chain (STO-3G, 1.8 bohr, Loewdin orbitals), eps = 1e-6, 16,384 walkers: the local energy
  after 64 rejection-free moves applied by Sherman-Morrison updates (Sec. III.B), before and after
  the periodic FP64 recompute of the tables;
- the uneven batch of Hubbard lattices 4x4 ... 10x10 (U/t = 4, half filling, periodic) and H40,
  H60, H100 chains, 2048 walkers each, in one persistent launch with the autotuned CTA width.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1807_10633_gb300 import systems as S
from tests.gpu_common import oracle_n

pytestmark = pytest.mark.gpu

NT = os.cpu_count() or 1


@pytest.fixture(scope="module")
def vmc():
    from paper_1807_10633_gb300 import vmc as v
    v.lib()
    return v


def _check_sample(sys_, prm, n, e_gpu, eps, idx):
    """n: (W, 2M) occupation numbers of the walkers whose GPU local energies are e_gpu."""
    orc = oracle.Oracle(sys_, prm)
    ref, _, _ = orc.local_energy_batch(np.ascontiguousarray(n[idx]), eps, n_threads=NT)
    err = np.max(np.abs(e_gpu[idx] - ref)) / sys_.n_elec
    assert err < 1e-4, err                                            # 0.1 mEh per electron
    return err


def test_h80_16384_walkers_64_moves_then_recompute(vmc):
    sys_ = S.named_system("H80")
    prm = S.make_params(sys_, seed=S.MASTER_SEED)
    W, eps = 16384, 1e-6
    occ = S.init_occupations(sys_, prm, W, seed=S.MASTER_SEED + 1)
    eng = vmc.Engine(sys_, prm, occ, eps=eps, precision=vmc.VMC_MIXED)
    idx = np.linspace(0, W - 1, 10).astype(int)
    try:
        vmc.Batch([eng]).autotune()
        for step in range(64):
            eng.local_energy()
            eng.ctmc_step(2024)
        e_moved = eng.local_energy()[0].cpu().numpy().copy()           # tables after 64 updates
        eng.refresh()                                                   # the periodic recompute
        e_fresh = eng.local_energy()[0].cpu().numpy().copy()
        eng.sync()
        n_now = eng.occupations()
    finally:
        eng.close()
    assert (n_now.sum(axis=1) == sys_.n_elec).all()
    err_moved = _check_sample(sys_, prm, n_now, e_moved, eps, idx)
    err_fresh = _check_sample(sys_, prm, n_now, e_fresh, eps, idx)
    print(f"H80 mixed after 64 moves: {1e3 * err_moved:.2e} mEh/e; after recompute {1e3 * err_fresh:.2e} mEh/e")


BATCH = [("hubbard4x4", 0.0), ("hubbard6x6", 0.0), ("hubbard8x8", 0.0), ("hubbard10x10", 0.0),
         ("H40", 1e-6), ("H60", 1e-6), ("H100", 1e-6)]


def test_uneven_batch_full_size(vmc):
    W = 2048
    engines, inputs = [], []
    try:
        for name, eps in BATCH:
            sys_ = S.named_system(name)
            prm = S.make_params(sys_, seed=S.MASTER_SEED)
            occ = S.init_occupations(sys_, prm, W, seed=S.MASTER_SEED + 1)
            engines.append(vmc.Engine(sys_, prm, occ, eps=eps, precision=vmc.VMC_MIXED))
            inputs.append((sys_, prm, occ, eps))
        b = vmc.Batch(engines)
        assert b.autotune() in (128, 256, 384, 512)
        b.local_energy()
        e = [x.e_loc.cpu().numpy().copy() for x in engines]
        for x in engines:
            x.sync()
    finally:
        for x in engines:
            x.close()
    idx = np.linspace(0, W - 1, 6).astype(int)
    for (sys_, prm, occ, eps), e_gpu in zip(inputs, e):
        _check_sample(sys_, prm, oracle_n(sys_, occ), e_gpu, eps, idx)
