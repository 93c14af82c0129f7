"""Edge cases and full-size configurations on the GPU (parity on sampled walkers)."""
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


def _check(vmc, sys_, prm, occ, eps, precision, idx=None, eps_run=None, tol=1e-10, gj32=0):
    eng = vmc.Engine(sys_, prm, occ, eps=eps, precision=precision)
    if gj32:   # mixed form with the FP32 Gauss-Jordan refresh instead of the FP64 LU
        vmc.vmc_set_option(eng.ctx, vmc.VMC_OPT_MIXED_REFRESH_GJ32, 1)
        eng.refresh()
    e, t = eng.local_energy(eps_run)
    eng.sync()
    e = e.cpu().numpy()
    idx = np.arange(len(occ)) if idx is None else idx
    orc = oracle.Oracle(sys_, prm)
    ref, _, _ = orc.local_energy_batch(oracle_n(sys_, occ[idx]), eps if eps_run is None else eps_run)
    eng.close()
    if precision == 0:
        assert rel_err(e[idx], ref) < tol
    else:
        assert np.max(np.abs(e[idx] - ref)) < 1e-4 * sys_.n_elec
    return e[idx], ref


def test_single_walker(vmc):
    sys_, prm, occ = make_case("H6", 1)
    _check(vmc, sys_, prm, occ, 1e-8, 0)


def test_odd_electron_counts(vmc):
    sys_ = S.hchain(7)          # 4 alpha + 3 beta
    prm = S.make_params(sys_, seed=2)
    occ = S.init_occupations(sys_, prm, 33, seed=3)
    _check(vmc, sys_, prm, occ, 1e-7, 0)


def test_eps_run_above_build_eps(vmc):
    sys_, prm, occ = make_case("H20", 64)
    _check(vmc, sys_, prm, occ, 1e-6, 0, eps_run=3e-4)


def test_large_eps_leaves_empty_lists(vmc):
    sys_, prm, occ = make_case("H20", 64)
    _check(vmc, sys_, prm, occ, 5e-2, 0)


def test_hubbard_2d_4x4(vmc):
    sys_, prm, occ = make_case("hubbard4x4", 129)
    _check(vmc, sys_, prm, occ, 0.0, 0)


@pytest.mark.parametrize("gj32", [0, 1], ids=["lu64", "gj32"])
def test_h80_mixed_form_mEh_per_particle(vmc, gj32):
    sys_, prm, occ = make_case("H80", 2048)
    e, ref = _check(vmc, sys_, prm, occ, 1e-6, 1, idx=np.arange(0, 2048, 97), gj32=gj32)
    print("H80 mixed max |dE| per particle (mEh):", 1e3 * np.max(np.abs(e - ref)) / sys_.n_elec)


def test_h80_fp64_form(vmc):
    sys_, prm, occ = make_case("H80", 2048)
    _check(vmc, sys_, prm, occ, 1e-6, 0, idx=np.arange(0, 2048, 131))


@pytest.mark.parametrize("precision,gj32", [(0, 0), (1, 0), (1, 1)], ids=["fp64", "mixed_lu64", "mixed_gj32"])
def test_tiny_leading_pivot_needs_a_row_exchange(vmc, precision, gj32):
    # C_alpha[0][0] = 1e-17 next to entries of order one: every walker that occupies alpha orbital 0
    # has C_occ^T[0][0] = 1e-17, which partial pivoting must move away from the diagonal; E_L (from
    # the G table) against the oracle's, whose LU is pinned against numpy determinants on this case
    sys_ = S.named_system("H20")
    prm = S.make_params(sys_, seed=11, j_scale=0.05, c_noise=0.1)
    occ = S.init_occupations(sys_, prm, 512, seed=12)
    occ = occ[occ[:, 0] == 0]                # the starts that occupy alpha orbital 0 (about 8 %)
    assert len(occ) >= 8
    prm.C_alpha[0, 0] = 1e-17
    _check(vmc, sys_, prm, occ, 1e-6, precision, gj32=gj32)
