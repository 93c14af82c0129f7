"""Failure detection on the GPU without a fault: a Slater block with an exactly singular C_occ (one
orbital coefficient column set to zero, so every walker's determinant is 0) is reported through the
latched status that vmc_sync returns, ln|psi| is -inf, the flag clears, and the same context goes on:
once the parameters are repaired, a table refresh gives tables whose local energies and residence
times equal those of an engine built on the good parameters from the start, bit for bit."""
import numpy as np
import pytest
import torch

from paper_1807_10633_gb300 import systems as S
from tests.gpu_common import make_case

pytestmark = pytest.mark.gpu

VMC_ERR_SINGULAR = 4


@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_singular_determinant_is_reported_and_a_refresh_recovers(form):
    from paper_1807_10633_gb300 import vmc
    lib = vmc.lib()
    precision = vmc.VMC_FP64 if form == "fp64" else vmc.VMC_MIXED
    sys_, prm, occ = make_case("H6", 16, j_scale=0.05, c_noise=0.1)
    bad = S.Params(prm.J.copy(), prm.C_alpha.copy(), prm.C_beta.copy())
    bad.C_alpha[:, 0] = 0.0            # column 0 of every walker's C_occ^alpha: det C_occ = 0 exactly

    eng = vmc.Engine(sys_, bad, occ, eps=1e-8, precision=precision)
    ref = vmc.Engine(sys_, prm, occ, eps=1e-8, precision=precision)
    try:
        assert lib.vmc_sync(eng.ctx) == VMC_ERR_SINGULAR
        assert lib.vmc_sync(eng.ctx) == 0                   # read once, then cleared
        lp = eng.log_psi()
        assert lib.vmc_sync(eng.ctx) == VMC_ERR_SINGULAR
        assert torch.isneginf(lp).all()

        eng.Ca.copy_(torch.from_numpy(prm.C_alpha))          # repair the parameters in place
        eng.refresh()
        assert lib.vmc_sync(eng.ctx) == 0
        e1, t1 = (x.cpu().numpy().copy() for x in eng.local_energy())
        e0, t0 = (x.cpu().numpy().copy() for x in ref.local_energy())
        assert lib.vmc_sync(eng.ctx) == 0 and lib.vmc_sync(ref.ctx) == 0
        assert np.isfinite(e1).all()
        np.testing.assert_array_equal(e1, e0)
        np.testing.assert_array_equal(t1, t0)
    finally:
        eng.close()
        ref.close()
