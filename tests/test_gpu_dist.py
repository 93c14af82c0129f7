"""Walker sharding through the library (the multi-GPU path, Sec. II.B: walkers are independent and
the walker sums of an iteration are the one exchange).

Two ranks of a gloo process group, both on cuda:0, each run the library's optimisation loop on their
own shard of the walkers; the all-reduce is the host-side collective, so no kernel of one rank ever
waits on the other.  Checked:
- the loop of two ranks against the oracle's loop over the same two shards, each shard sampled with
  its rank's Philox seed word: the energy of Eq. (vmc) of every iteration and every parameter after
  every AMSGrad step (FP64 form, CTMC choices bit-exact, so both visit the same determinants), and
  bit-identical parameter replicas on the two ranks;
- bench.py under torchrun with two ranks: its two-graph step with the exchange between the graphs
  runs, rank 0 alone prints the JSON line, and the replicas stay identical."""
import json
import os
import socket
import subprocess
import sys
from pathlib import Path
from types import SimpleNamespace

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_1807_10633_gb300 import dist as D
from tests.gpu_common import make_case, oracle_n, rel_err

pytestmark = pytest.mark.gpu

ROOT = Path(__file__).resolve().parents[1]
CASE = dict(name="H4", W=96, eps=1e-8, n_iter=5, sweeps=3, seed=99, warm=2)
WORLD = 2


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _split(p, M, na, nb):
    N2 = 2 * M
    a, b = N2 * N2, N2 * N2 + M * na
    return p[:a].reshape(N2, N2), p[a:b].reshape(M, na), p[b:b + M * nb].reshape(M, nb)


def _rank(rank, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        from paper_1807_10633_gb300 import optimize as O
        from paper_1807_10633_gb300 import vmc
        vmc.lib()
        c = CASE
        sys_, prm, occ = make_case(c["name"], c["W"], j_scale=0.05, c_noise=0.1)
        s0, cnt = D.walker_shard(c["W"], rank, WORLD)
        eng = vmc.Engine(sys_, prm, occ[s0:s0 + cnt], eps=c["eps"], precision=vmc.VMC_FP64)
        seen = []
        try:
            its = O.optimize(eng, c["n_iter"], c["sweeps"], seed=c["seed"], warm=c["warm"],
                             callback=lambda it: seen.append(eng.p.cpu().numpy().copy()))
        finally:
            eng.close()
        out[rank] = ([it.energy for it in its], seen)
    finally:
        dist.destroy_process_group()


def _oracle_sharded_loop():
    """The loop of Sec. II.C from the oracle's pieces, the walkers split as the ranks split them:
    shard r is sampled with the Philox key (rank seed word of r, index within the shard), and the
    sums of all shards form one gradient per iteration (Eq. grad), then one AMSGrad step."""
    c = CASE
    sys_, prm, occ = make_case(c["name"], c["W"], j_scale=0.05, c_noise=0.1)
    M, na, nb = sys_.M, sys_.n_alpha, sys_.n_beta
    shards = []
    for r in range(WORLD):
        s0, cnt = D.walker_shard(c["W"], r, WORLD)
        shards.append([np.ascontiguousarray(oracle_n(sys_, occ[s0:s0 + cnt])), np.zeros(cnt, dtype=np.uint64)])
    p = prm.flat().astype(np.float64).copy()
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    energies, params = [], []
    for k in range(c["n_iter"]):
        J, Ca, Cb = _split(p, M, na, nb)
        orc = oracle.Oracle(sys_, SimpleNamespace(J=J.copy(), C_alpha=Ca.copy(), C_beta=Cb.copy()))
        AO = np.zeros_like(p)
        AEO = np.zeros_like(p)
        aoJ, aoA, aoB = (np.ascontiguousarray(x) for x in _split(AO, M, na, nb))
        aeJ, aeA, aeB = (np.ascontiguousarray(x) for x in _split(AEO, M, na, nb))
        T = TE = 0.0
        for r, (n, ctr) in enumerate(shards):
            for _ in range(c["sweeps"]):
                before = n.copy()
                el, tr, _, err = orc.sweep(n, c["eps"], D.rank_seed(c["seed"] + k, r), ctr)
                assert err == 0
                for w in range(n.shape[0]):
                    orc.grad_logpsi(before[w], tr[w], aoJ, aoA, aoB)
                    orc.grad_logpsi(before[w], tr[w] * el[w], aeJ, aeA, aeB)
                T += tr.sum()
                TE += (tr * el).sum()
        AO = np.concatenate([aoJ.ravel(), aoA.ravel(), aoB.ravel()])
        AEO = np.concatenate([aeJ.ravel(), aeA.ravel(), aeB.ravel()])
        g = 2.0 * (AEO / T - (TE / T) * (AO / T))
        oracle.amsgrad(p, g, m, v, 0.001 if k < c["warm"] else 0.01, 0.1, 0.01)
        energies.append(TE / T)
        params.append(p.copy())
    return np.array(energies), params


def test_two_rank_optimisation_loop_matches_the_sharded_oracle_loop():
    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:   # no fork of a process that may hold a CUDA context
        out = mgr.dict()
        mp.spawn(_rank, args=(port, out), nprocs=WORLD, join=True)
        res = dict(out)
    ref_e, ref_p = _oracle_sharded_loop()
    (e0, p0), (e1, p1) = res[0], res[1]
    assert e0 == e1                                    # both ranks see the reduced sums
    assert rel_err(e0, ref_e) < 1e-10
    for k in range(CASE["n_iter"]):
        np.testing.assert_array_equal(p0[k], p1[k])    # identical replicas
        assert np.max(np.abs(p0[k] - ref_p[k])) < 1e-10, f"iteration {k}"


def test_bench_two_ranks_one_exchange_per_step():
    env = dict(os.environ, MASTER_ADDR="127.0.0.1", VMC_DIST_BACKEND="gloo")
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
                        "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), str(ROOT / "bench.py"),
                        "--gpus", "2", "--system", "H20", "--walkers", "512", "--steps", "2", "--warmup", "3",
                        "--repeats", "1", "--forms", "mixed", "--no-cpu-baseline", "--no-batch"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [json.loads(x) for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    line = lines[0]
    assert line["n_gpus"] == 2 and line["value"] > 0 and line["e2e"]["value"] > 0
    assert line["replicas_identical"] is True
    assert "gloo" in line["config"]["parallelism"]
    assert line["gpu_launches"] > 0
