"""Batched launches over systems of uneven size reproduce the per-system calls (needs a GB300)."""
import numpy as np
import pytest
import torch

from tests.gpu_common import make_case

pytestmark = pytest.mark.gpu

CASES = [("hubbard4x4", 150), ("H20", 200), ("hubbard6x6", 100), ("H12", 64)]


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_sweeps_match_per_system_sweeps(precision):
    from paper_1807_10633_gb300 import vmc
    eps = {"hubbard4x4": 0.0, "hubbard6x6": 0.0, "H20": 1e-6, "H12": 1e-6}
    single, batched = [], []
    for name, W in CASES:
        sys_, prm, occ = make_case(name, W)
        single.append(vmc.Engine(sys_, prm, occ, eps=eps[name], precision=precision))
        batched.append(vmc.Engine(sys_, prm, occ, eps=eps[name], precision=precision))
    b = vmc.Batch(batched)
    for step in range(6):
        if step == 3:
            assert b.autotune() in (128, 256, 384, 512)
        for e in single:
            e.local_energy()
            e.ctmc_step(17)
        b.local_energy()
        b.ctmc_step(17)
        torch.cuda.synchronize()
        for e1, e2 in zip(single, batched):
            assert torch.equal(e1.e_loc, e2.e_loc), step
            assert torch.equal(e1.t_res, e2.t_res), step
            assert torch.equal(e1.moves, e2.moves), step
    for e1, e2 in zip(single, batched):
        assert np.array_equal(e1.occupations(), e2.occupations())
        e1.sync(); e2.sync()
    for e in single + batched:
        e.close()
