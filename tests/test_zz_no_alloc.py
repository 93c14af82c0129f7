"""The allocation-free gradient entry point agrees with vmc_grad_logpsi (needs a GB300).

vmc_grad_logpsi_noalloc serves callers that may not allocate device memory: services whose device
memory belongs to another allocator's pool, deployments whose footprint is fixed up front, and host
loops that must not stall on the synchronisation an allocation may cause.  It keeps its scratch in a
fixed device array inside the library.  This file is collected last so that a failure here comes
after every other test has run.
"""
import ctypes as ct

import numpy as np
import pytest
import torch

from tests.gpu_common import make_case

pytestmark = pytest.mark.gpu


def _free_bytes() -> int:
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


# 1,000 walkers: one walker chunk for the Jastrow and orbital partials; 5,000 walkers: several
# chunks of each (more than 1,024 and 256 walkers), so the chunked partial layout is exercised
@pytest.mark.parametrize("W", [1000, 5000])
@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-5)])
def test_noalloc_vjp_matches_context_vjp_on_two_calls(precision, tol, W):
    from paper_1807_10633_gb300 import vmc
    sys_, prm, occ = make_case("H20", W)
    eng = vmc.Engine(sys_, prm, occ, eps=1e-6, precision=precision)
    stream = torch.cuda.current_stream()
    ws = eng.walkers.struct()
    rng = np.random.default_rng(11)
    ws_all = [torch.tensor(rng.normal(size=eng.W), device="cuda") for _ in range(2)]
    refs = [tuple(torch.zeros_like(x) for x in (eng.J, eng.Ca, eng.Cb)) for _ in range(2)]
    gots = [tuple(torch.zeros_like(x) for x in (eng.J, eng.Ca, eng.Cb)) for _ in range(2)]
    # set-up call: looks up the scratch address and loads the kernels; later calls allocate nothing
    warm = tuple(torch.zeros_like(x) for x in (eng.J, eng.Ca, eng.Cb))
    vmc.vmc_grad_logpsi_noalloc(ws, ws_all[0], *warm, stream=stream)
    reserved = torch.cuda.memory_reserved()
    for call in range(2):
        w = ws_all[call]
        eng.grad_logpsi(w, *refs[call])
        free0 = _free_bytes()
        vmc.vmc_grad_logpsi_noalloc(ws, w, *gots[call], stream=stream)
        assert _free_bytes() == free0, "the entry point changed the device's free memory"
        assert torch.cuda.memory_reserved() == reserved
        scale = float(w.abs().sum())
        for a, b in zip(gots[call], refs[call]):
            err = (a - b).abs().max().item()
            assert err <= tol * scale * max(1.0, b.abs().max().item()), (call, err)
        eng.local_energy()
        eng.ctmc_step(5 + call)          # move the walkers so the second call sees new tables
    eng.sync()
    eng.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1807_10633_gb300 import vmc
    sys_, prm, occ = make_case("H6", 16)
    eng = vmc.Engine(sys_, prm, occ, eps=1e-6, precision=0)
    big = 2_100_000                      # 8 W bytes of fixed-point weights alone exceed 16 MiB
    w = torch.zeros(big, dtype=torch.float64, device="cuda")
    ws = eng.walkers.struct()
    ws.W = big
    out = tuple(torch.zeros_like(x) for x in (eng.J, eng.Ca, eng.Cb))
    with pytest.raises(vmc.VmcError, match="ERR_ARG"):
        vmc.vmc_grad_logpsi_noalloc(ws, w, *out)
    ws = eng.walkers.struct()
    ws.n_alpha = ws.n_beta = 0           # no electrons: nothing to size the orbital block by
    st = vmc.lib().vmc_grad_logpsi_noalloc(ct.byref(ws), w.data_ptr(), *(x.data_ptr() for x in out), None)
    assert st == 1
    torch.cuda.synchronize()
    assert all(float(x.abs().sum()) == 0.0 for x in out)   # nothing was launched
    eng.close()
