"""Checkpoint and resume of the optimisation loop on the GPU: six AMSGrad iterations in one run
against three, a checkpoint written to disk, a new engine rebuilt from it, and three more.  The
energies of every iteration, the final parameters and the final occupations must be bit-identical
(FP64 and mixed forms, with and without a correlator product)."""
import numpy as np
import pytest
import torch

from paper_1807_10633_gb300 import checkpoint as C
from paper_1807_10633_gb300 import optimize as O
from paper_1807_10633_gb300 import systems as S
from tests.gpu_common import make_case

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("form,with_cps", [("fp64", False), ("mixed", False), ("mixed", True)])
def test_resume_continues_bit_identically(tmp_path, form, with_cps):
    from paper_1807_10633_gb300 import vmc
    vmc.lib()
    precision = vmc.VMC_FP64 if form == "fp64" else vmc.VMC_MIXED
    sys_, prm, occ = make_case("H6", 64, j_scale=0.05, c_noise=0.1)
    cps = S.make_cps(sys_, seed=5, noise=0.05) if with_cps else None
    run = dict(sweeps=3, seed=41, warm=2)

    eng = vmc.Engine(sys_, prm, occ, eps=1e-8, precision=precision, cps=cps)
    try:
        ref = O.optimize(eng, 6, **run)
        p_ref = eng.p.cpu().numpy().copy()
        occ_ref = eng.walkers.occ_list.cpu().numpy().copy()
    finally:
        eng.close()

    eng1 = vmc.Engine(sys_, prm, occ, eps=1e-8, precision=precision, cps=cps)
    try:
        st = O.OptState.fresh(eng1)
        first = O.optimize(eng1, 3, state=st, **run)
        assert st.next_iter == 3
        path = C.save(tmp_path / "run.ckpt", eng1, st, sys_)
    finally:
        eng1.close()

    eng2, st2 = C.load(path, sys_)
    try:
        assert st2.next_iter == 3
        second = O.optimize(eng2, 3, state=st2, **run)
        got = [it.energy for it in first + second]
        assert got == [it.energy for it in ref]
        assert [it.index for it in second] == [3, 4, 5]
        np.testing.assert_array_equal(eng2.p.cpu().numpy(), p_ref)
        np.testing.assert_array_equal(eng2.walkers.occ_list.cpu().numpy(), occ_ref)
    finally:
        eng2.close()
    torch.cuda.synchronize()
