"""Multi-process host logic of walker sharding (world size 2, gloo on the CPU): the shards cover the
walkers exactly once, rank seeds differ, the single all-reduce adds every rank's walker sums, and
the AMSGrad update of the reduced gradient leaves identical parameters on every rank; a rank that
leaves or stalls between steps makes the other rank's exchange end with an error, not a hang."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1807_10633_gb300 import dist as D


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _amsgrad(p, g, m, v, alpha, b1, b2):
    # Eqs. (m1)-(m2) as printed: m <- (1 - b1) m + b1 g, v <- max(v, (1 - b2) v + b2 g^2)
    m[:] = (1 - b1) * m + b1 * g
    v[:] = np.maximum(v, (1 - b2) * v + b2 * g * g)
    nz = v > 0
    p[nz] -= alpha * m[nz] / np.sqrt(v[nz])


def _worker(rank, world, port, n_params, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        red, ao, aeo, sums = D.sums_buffer(n_params, "cpu")
        rng = np.random.default_rng(100 + rank)        # this rank's walker sums
        ao.copy_(torch.tensor(rng.normal(size=n_params)))
        aeo.copy_(torch.tensor(rng.normal(size=n_params)))
        sums.copy_(torch.tensor([1.0 + rank, -0.5 * (1.0 + rank)]))
        D.allreduce_sums(red)
        T, E = float(sums[0]), float(sums[1] / sums[0])
        g = 2.0 * (aeo.numpy() / T - E * ao.numpy() / T)   # Eq. (grad) from the reduced sums
        p = np.linspace(-1, 1, n_params); m = np.zeros(n_params); v = np.zeros(n_params)
        _amsgrad(p, g, m, v, 0.01, 0.1, 0.01)
        out[rank] = (red.numpy().copy(), p, D.walker_shard(1001, rank, world), D.rank_seed(1807, rank))
    finally:
        dist.destroy_process_group()


def test_two_rank_gradient_exchange():
    world, n_params = 2, 257
    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:   # no fork of a process that may hold a CUDA context
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, n_params, out), nprocs=world, join=True)
        res = dict(out)
    expect = np.zeros(2 * n_params + 2)
    for r in range(world):
        rng = np.random.default_rng(100 + r)
        expect[:n_params] += rng.normal(size=n_params)
        expect[n_params:2 * n_params] += rng.normal(size=n_params)
        expect[2 * n_params:] += [1.0 + r, -0.5 * (1.0 + r)]
    for r in range(world):
        np.testing.assert_allclose(res[r][0], expect, rtol=1e-14, atol=1e-14)
    np.testing.assert_array_equal(res[0][1], res[1][1])      # identical parameter replicas
    (s0, c0), (s1, c1) = res[0][2], res[1][2]
    assert s0 == 0 and s0 + c0 == s1 and s1 + c1 == 1001
    assert res[0][3] != res[1][3]


@pytest.mark.parametrize("W,world", [(0, 3), (7, 1), (7, 8), (32768, 8), (1001, 7)])
def test_walker_shard_partition(W, world):
    seen = np.zeros(W, dtype=int)
    for r in range(world):
        s, c = D.walker_shard(W, r, world)
        seen[s:s + c] += 1
        assert c in (W // world, W // world + 1)
    assert (seen == 1).all()
    with pytest.raises(ValueError):
        D.walker_shard(W, world, world)


def _failing_worker(rank, world, port, mode, out):
    import datetime
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=3))
    try:
        red, _, _, sums = D.sums_buffer(8, "cpu")
        sums.fill_(1.0)
        if rank == 1:
            if mode == "exits":
                return                       # leaves between steps, before the exchange
            import time
            time.sleep(6)                    # stalls past the process-group timeout
            return
        try:
            D.allreduce_sums(red)
            out[rank] = "completed"
        except RuntimeError as e:            # the exchange ends with an error instead of hanging
            out[rank] = "error: " + str(e)[:80]
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("mode", ["exits", "stalls"])
def test_a_rank_that_leaves_ends_the_exchange_with_an_error(mode):
    """A rank that leaves (or stops answering) between steps: the other rank's all-reduce of the
    walker sums raises within the process-group timeout instead of waiting for ever."""
    import time
    port = _free_port()
    t0 = time.monotonic()
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_failing_worker, args=(2, port, mode, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0].startswith("error"), res
    assert time.monotonic() - t0 < 60
