"""The optimisation loop of the method (Sec. II.C): every iteration samples the wavefunction with
`sweeps` rejection-free CTMC steps of all walkers (Sec. II.B), accumulates the residence-time
weighted sums of Eq. (vmc) and the gradient pieces of Eq. (grad), forms the energy gradient
g = 2 (<E_L O> - <E_L><O>), applies one AMSGrad step (Eqs. m1-m2, beta1 = 0.1, beta2 = 0.01) and
recomputes the walker tables for the new parameters.  The step size starts at 0.001 and is raised to
0.01 after the first iterations, as in the paper's hydrogen-chain runs (Sec. IV.B).

Orchestration only: every step runs in the CUDA library through its C ABI.
"""
from __future__ import annotations

import time
from dataclasses import dataclass

import torch

from . import dist as D
from . import vmc


@dataclass
class Iteration:
    index: int
    alpha: float
    energy: float              # sum t E_L / sum t over the iteration's samples (Eq. vmc)
    energy_per_electron: float
    t_sum: float
    grad_norm: float
    ms: float                  # device time of the iteration (CUDA events)
    rate_overflow: bool = False   # a CTMC rate reached the fixed-point limit in this iteration


RATE_OVERFLOW = 6      # VMC_ERR_OVERFLOW


@dataclass
class OptState:
    """The AMSGrad moments m and v (Eqs. m1-m2) and the index of the next iteration: with the
    parameters and the walkers, what an interrupted optimisation needs to go on (checkpoint.py)."""
    m: torch.Tensor
    v: torch.Tensor
    next_iter: int = 0

    @classmethod
    def fresh(cls, eng: vmc.Engine) -> "OptState":
        z = torch.zeros(eng.n_params, dtype=torch.float64, device=eng.p.device)
        return cls(z, z.clone(), 0)


def alpha_schedule(k: int, alpha0: float = 0.001, alpha1: float = 0.01, warm: int = 5) -> float:
    """Step size of iteration k: alpha0 for the first `warm` iterations, then alpha1."""
    return alpha0 if k < warm else alpha1


def optimize(eng: vmc.Engine, n_iter: int, sweeps: int, seed: int = 1807, burn_in: int = 0,
             alpha0: float = 0.001, alpha1: float = 0.01, warm: int = 5, beta1: float = 0.1,
             beta2: float = 0.01, n_elec: int | None = None, callback=None,
             train_jastrow: bool = True, state: OptState | None = None) -> list[Iteration]:
    """Run n_iter AMSGrad iterations on `eng` (its parameters eng.p are updated in place).

    state: the AMSGrad moments and the index of the first iteration (None: zero moments, iteration
    0); it is updated in place, so a later call with the same state continues the run (the step
    size schedule and the CTMC seeds follow the global iteration index).

    Each iteration: `sweeps` CTMC steps; the first `burn_in` of them move the walkers without
    entering the sums.  Under an initialised process group the walker sums of all ranks are added
    before the gradient is formed, so every rank applies the same update.

    A CTMC rate at or above the fixed-point limit 2^43 (a walker on a near-node determinant of the
    current wavefunction, whose neighbour has a ratio that large) is clamped by the library and
    reported through the latched VMC_ERR_OVERFLOW; such a walker's residence time is below 2^-43,
    so its weight in the sums is nil.  The loop records the event in the iteration and continues;
    every other latched error is raised.

    train_jastrow=False keeps the pair-Jastrow block fixed: the energy gradient and the AMSGrad
    step cover the Slater coefficients and correlator coefficients only (the flat parameters are
    [J | C_alpha | C_beta | correlators], so this is the tail of the buffers).
    """
    if sweeps <= burn_in:
        raise ValueError("sweeps must exceed burn_in")
    dev = eng.p.device
    stream = torch.cuda.current_stream(dev)
    np_ = eng.n_params
    red, AO, AEO, sums = D.sums_buffer(np_, dev)
    g = torch.zeros(np_, dtype=torch.float64, device=dev)
    st = state if state is not None else OptState.fresh(eng)
    if st.m.numel() != np_ or st.v.numel() != np_:
        raise ValueError("optimiser state does not match the engine's parameters")
    m, v = st.m, st.v
    AOv, AEOv = eng.split(AO), eng.split(AEO)
    AOc, AEOc = eng.split_cps(AO), eng.split_cps(AEO)   # correlator coefficients (None without them)
    ne = n_elec or (eng.na + eng.nb)
    rank = 0
    if torch.distributed.is_available() and torch.distributed.is_initialized():
        rank = torch.distributed.get_rank()
    out = []
    for k in range(st.next_iter, st.next_iter + n_iter):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        red.zero_()
        ws = eng.walkers.struct()
        prm = eng.params
        for s in range(sweeps):
            vmc.vmc_local_energy(eng.ctx, eng.lists, prm, ws, eng.eps, eng.e_loc, eng.t_res)
            if s >= burn_in:
                vmc.vmc_accumulate_gradient(eng.ctx, ws, eng.t_res, eng.e_loc, AOv, AEOv, sums)
                if AOc is not None:
                    vmc.vmc_accumulate_gradient_cps(eng.ctx, ws, prm, eng.t_res, eng.e_loc, AOc, AEOc)
            vmc.vmc_ctmc_step(eng.ctx, eng.lists, prm, ws, D.rank_seed(seed + k, rank), eng.moves)
        D.allreduce_sums(red)
        alpha = alpha_schedule(k, alpha0, alpha1, warm)
        j0 = 0 if train_jastrow else (2 * eng.M) ** 2
        vmc.vmc_energy_gradient(eng.ctx, sums, AO[j0:], AEO[j0:], g[j0:])
        vmc.vmc_amsgrad_update(eng.ctx, eng.p[j0:], g[j0:], m[j0:], v[j0:], alpha, beta1, beta2)
        vmc.vmc_walkers_refresh(eng.ctx, eng.lists, prm, ws)
        b.record(stream)
        rc = vmc.lib().vmc_sync(eng.ctx)             # waits for the stream, returns and clears the flags
        if rc not in (0, RATE_OVERFLOW):
            vmc._check(eng.ctx, rc)
        T, TE = (float(x) for x in sums.cpu())
        it = Iteration(k, alpha, TE / T, TE / T / ne, T, float(g.norm()), a.elapsed_time(b), rc == RATE_OVERFLOW)
        st.next_iter = k + 1
        out.append(it)
        if callback is not None:
            callback(it)
    return out


def parser():
    import argparse

    from . import systems as S
    ap = argparse.ArgumentParser(description="AMSGrad optimisation of a Jastrow-Slater wavefunction on one GPU")
    ap.add_argument("--system", default="H20")
    ap.add_argument("--walkers", type=int, default=4096)
    ap.add_argument("--sweeps", type=int, default=16)
    ap.add_argument("--burn-in", type=int, default=0)
    ap.add_argument("--iters", type=int, default=30)
    ap.add_argument("--eps", type=float, default=1e-6)
    ap.add_argument("--form", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--seed", type=int, default=S.MASTER_SEED)
    ap.add_argument("--alpha0", type=float, default=0.001, help="step size of the first --warm iterations")
    ap.add_argument("--alpha1", type=float, default=0.01, help="step size afterwards")
    ap.add_argument("--warm", type=int, default=5)
    ap.add_argument("--checkpoint", default="",
                    help="write a checkpoint to this file at the end (and every --checkpoint-every iterations)")
    ap.add_argument("--checkpoint-every", type=int, default=0)
    ap.add_argument("--resume", default="",
                    help="continue from this checkpoint (same --system; its form, eps and walkers are kept)")
    return ap


def main(argv=None):
    import json

    from . import checkpoint as C
    from . import systems as S
    args = parser().parse_args(argv)
    sys_ = S.named_system(args.system)
    if args.resume:
        eng, st = C.load(args.resume, sys_)
    else:
        prm = S.make_params(sys_, seed=args.seed)
        occ = S.init_occupations(sys_, prm, args.walkers, seed=args.seed + 1)
        eng = vmc.Engine(sys_, prm, occ, eps=args.eps,
                         precision=vmc.VMC_MIXED if args.form == "mixed" else vmc.VMC_FP64)
        st = OptState.fresh(eng)
    vmc.Batch([eng]).autotune()
    t0 = time.perf_counter()
    its = []
    chunk = args.checkpoint_every if args.checkpoint and args.checkpoint_every > 0 else max(1, args.iters)
    left = args.iters
    while left > 0:   # chunks of one run: the state carries the schedule and the seeds across them
        k = min(chunk, left)
        its += optimize(eng, k, args.sweeps, seed=args.seed, burn_in=args.burn_in, n_elec=sys_.n_elec,
                        alpha0=args.alpha0, alpha1=args.alpha1, warm=args.warm, state=st,
                        callback=lambda it: print(json.dumps(it.__dict__), flush=True))
        left -= k
        if args.checkpoint:
            C.save(args.checkpoint, eng, st, sys_)
    form = "fp64" if eng.walkers.precision == vmc.VMC_FP64 else "mixed"
    print(json.dumps({"system": args.system, "walkers": eng.W, "sweeps": args.sweeps, "form": form,
                      "eps": eng.eps, "wall_s": time.perf_counter() - t0, "next_iter": st.next_iter,
                      "first": its[0].energy_per_electron if its else None,
                      "last": its[-1].energy_per_electron if its else None}))
    eng.close()


if __name__ == "__main__":
    main()
