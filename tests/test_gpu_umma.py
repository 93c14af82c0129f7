"""Tensor-core (tcgen05, 3xTF32) G refresh agrees with the CUDA-core refresh (needs a GB300)."""
import numpy as np
import pytest
import torch

from paper_1807_10633_gb300 import systems as S
from tests.gpu_common import make_case

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,W", [("H20", 77), ("H80", 300), ("H7", 40), ("hubbard6x6", 50)])
def test_tensor_core_G_matches_cuda_core_G(name, W):
    from paper_1807_10633_gb300 import vmc
    if name == "H7":
        sys_ = S.hchain(7)
        prm = S.make_params(sys_, seed=2)
        occ = S.init_occupations(sys_, prm, W, seed=3)
    else:
        sys_, prm, occ = make_case(name, W)
    eng = vmc.Engine(sys_, prm, occ, eps=1e-6, precision=vmc.VMC_MIXED)
    vmc.vmc_set_option(eng.ctx, vmc.VMC_OPT_G_TENSOR_CORES, 0)
    eng.init()
    eng.sync()
    g_cuda = eng.walkers.G.clone()
    vmc.vmc_set_option(eng.ctx, vmc.VMC_OPT_G_TENSOR_CORES, 1)
    eng.init()
    eng.sync()
    g_tc = eng.walkers.G.clone()
    scale = g_cuda.abs().max().item()
    assert (g_tc - g_cuda).abs().max().item() <= 2e-5 * max(1.0, scale)
    eng.close()
