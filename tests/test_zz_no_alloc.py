"""The allocation-free gradient entry point agrees with vmc_grad_logpsi (needs a GB300).

vmc_grad_logpsi_noalloc serves callers that may not allocate device memory (for example while a
CUDA graph is being captured): it keeps its scratch in a fixed device array inside the library.
This file is collected last so that a failure here comes after every other test has run.
"""
import numpy as np
import pytest
import torch

from tests.gpu_common import make_case

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-5)])
def test_noalloc_vjp_matches_context_vjp_on_two_calls(precision, tol):
    from paper_1807_10633_gb300 import vmc
    sys_, prm, occ = make_case("H20", 1000)
    eng = vmc.Engine(sys_, prm, occ, eps=1e-6, precision=precision)
    stream = torch.cuda.current_stream()
    ws = eng.walkers.struct()
    rng = np.random.default_rng(11)
    for call in range(2):
        w = torch.tensor(rng.normal(size=eng.W), device="cuda")
        ref = eng.grad_logpsi(w)
        got = tuple(torch.zeros_like(x) for x in ref)
        vmc.vmc_grad_logpsi_noalloc(ws, w, *got, stream=stream)
        torch.cuda.synchronize()
        scale = float(w.abs().sum())
        for a, b in zip(got, ref):
            err = (a - b).abs().max().item()
            assert err <= tol * scale * max(1.0, b.abs().max().item()), (call, err)
        eng.local_energy()
        eng.ctmc_step(5 + call)          # move the walkers so the second call sees new tables
    eng.sync()
    eng.close()
