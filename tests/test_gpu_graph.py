"""A CTMC sweep captured in a CUDA graph replays exactly like the eager calls (needs a GB300)."""
import numpy as np
import pytest
import torch

from tests.gpu_common import make_case

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_replay_matches_eager(precision):
    from paper_1807_10633_gb300 import vmc
    sys_, prm, occ = make_case("H20", 300)
    engines = [vmc.Engine(sys_, prm, occ, eps=1e-6, precision=precision) for _ in range(2)]
    eager, graphed = engines
    # warm-up call on the graphed engine so every workspace exists before capture
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        vmc.vmc_set_stream(graphed.ctx, s)
        graphed.local_energy()
        graphed.ctmc_step(3)
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            graphed.local_energy()
            graphed.ctmc_step(3)
    torch.cuda.current_stream().wait_stream(s)
    eager.local_energy()
    eager.ctmc_step(3)
    for step in range(5):
        e1, t1 = eager.local_energy()
        m1 = eager.ctmc_step(3).clone()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(e1, graphed.e_loc), step
        assert torch.equal(t1, graphed.t_res), step
        assert torch.equal(m1, graphed.moves), step
    assert np.array_equal(eager.occupations(), graphed.occupations())
    for e in engines:
        e.sync()
        e.close()
