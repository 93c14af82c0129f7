"""Walker sharding across GPUs (one process per GPU) and the one exchange of an optimisation step.

Walkers are independent for the local energy, the CTMC moves and the table updates (Sec. II.B);
the only quantities that couple them are the walker sums of one optimisation iteration,
(sum t, sum t E_L, sum t O_k, sum t E_L O_k) of Eq. (vmc), from which the energy gradient is
formed.  Each rank therefore runs its own walkers and sums, the sums are added across ranks by
one all-reduce of a single flat buffer, and every rank then applies the same AMSGrad update to its
replica of the parameters, which stay identical on all ranks.
"""
from __future__ import annotations

import torch


def walker_shard(w_total: int, rank: int, world: int) -> tuple[int, int]:
    """(first walker, walker count) of `rank`: contiguous blocks, the first w_total % world ranks
    one walker longer."""
    if world < 1 or not 0 <= rank < world or w_total < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(w_total, world)
    start = rank * base + min(rank, extra)
    return start, base + (1 if rank < extra else 0)


def rank_seed(seed: int, rank: int) -> int:
    """CTMC seed of `rank`.  The Philox key is (seed, local walker index); giving every rank its own
    seed word keeps all (rank, walker) streams distinct."""
    return (int(seed) ^ (int(rank) << 40)) & 0xFFFFFFFFFFFFFFFF


def sums_buffer(n_params: int, device) -> tuple[torch.Tensor, torch.Tensor, torch.Tensor, torch.Tensor]:
    """One flat FP64 buffer [A_O (n_params) | A_EO (n_params) | sum t, sum t E_L] and its three views,
    so that the exchange is a single collective."""
    red = torch.zeros(2 * n_params + 2, dtype=torch.float64, device=device)
    return red, red[:n_params], red[n_params:2 * n_params], red[2 * n_params:]


def allreduce_sums(red: torch.Tensor, group=None) -> torch.Tensor:
    """Add the walker sums of every rank (in place); a no-op without an initialised process group."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(red, op=dist.ReduceOp.SUM, group=group)
    return red
