"""The paper's two studies of Sec. IV on synthetic STO-3G hydrogen chains, run on one GPU.

* ``eps_protocol`` (Sec. IV.A, Table II): optimise the wavefunction with a loose screening
  threshold, then evaluate the energy of the optimised wavefunction with tighter thresholds (the
  CTMC move set and E_L both use the evaluation threshold), reporting the energy per electron with
  a blocking error bar and the cost per 1000 samples at every threshold.
* ``chain_optimisation`` (Sec. IV.B, Fig. 2): AMSGrad optimisation of chains of growing length at
  the same number of samples per iteration and the same step-size schedule, recording the energy
  per electron of every iteration.

Samples come from long CTMC chains, as in the paper's runs (a few thousand walkers, each moved for
many sweeps per iteration after a short burn-in), rather than from many short chains.

Orchestration only: every step runs in the CUDA library through its C ABI.
"""
from __future__ import annotations

import json
import math
import time

import numpy as np
import torch

from . import optimize as O
from . import systems as S
from . import vmc


def blocking_error(e: np.ndarray, t: np.ndarray, block: int) -> tuple[float, float]:
    """Residence-time-weighted mean of per-sweep samples e[s, w] (weights t[s, w]) and its standard
    error from means over blocks of `block` consecutive sweeps (all walkers of a block together)."""
    n_s = e.shape[0] // block
    if n_s < 2:
        raise ValueError("need at least two blocks")
    E = float((t * e).sum() / t.sum())
    bm = np.array([(t[k * block:(k + 1) * block] * e[k * block:(k + 1) * block]).sum()
                   / t[k * block:(k + 1) * block].sum() for k in range(n_s)])
    return E, float(bm.std(ddof=1) / math.sqrt(n_s))


def sample_energy(eng: vmc.Engine, eps_run: float, sweeps: int, burn_in: int, seed: int, block: int = 8):
    """Energy of the engine's wavefunction at threshold eps_run: `burn_in` CTMC sweeps, then
    `sweeps` sweeps whose (E_L, t) of every walker are kept.  Returns (energy, error, ms per sweep)."""
    stream = torch.cuda.current_stream(eng.device)
    ws, prm = eng.walkers.struct(), eng.params
    for s in range(burn_in):
        vmc.vmc_local_energy(eng.ctx, eng.lists, prm, ws, eps_run, eng.e_loc, eng.t_res)
        vmc.vmc_ctmc_step(eng.ctx, eng.lists, prm, ws, seed + s, eng.moves)
    E = torch.zeros((sweeps, eng.W), dtype=torch.float64, device=eng.device)
    T = torch.zeros_like(E)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for s in range(sweeps):
        vmc.vmc_local_energy(eng.ctx, eng.lists, prm, ws, eps_run, eng.e_loc, eng.t_res)
        E[s].copy_(eng.e_loc)
        T[s].copy_(eng.t_res)
        vmc.vmc_ctmc_step(eng.ctx, eng.lists, prm, ws, seed + burn_in + s, eng.moves)
    b.record(stream)
    eng.sync()
    e, err = blocking_error(E.cpu().numpy(), T.cpu().numpy(), block)
    return e, err, a.elapsed_time(b) / sweeps


def eps_protocol(name: str = "H20", eps_opt: float = 1e-4, eps_eval=(1e-4, 1e-5, 1e-6, 0.0), walkers: int = 2048,
                 sweeps: int = 64, burn_in: int = 4, iters: int = 40, eval_sweeps: int = 256,
                 seed: int = S.MASTER_SEED, form: int = vmc.VMC_MIXED, cps: bool = False,
                 start: str = "core") -> dict:
    """Optimise at eps_opt, then evaluate the optimised wavefunction at every eps in eps_eval.
    cps: 5-site correlators x Slater with the pair Jastrow zero and fixed (the paper's form)."""
    sys_ = S.named_system(name)
    prm = S.make_params(sys_, seed=seed, start=start, c_noise=0.01 if start == "core" else 0.05)
    corr = None
    if cps:
        prm.J[:] = 0.0
        corr = S.make_cps(sys_, seed=seed + 7, noise=0.0)
    occ = S.init_occupations(sys_, prm, walkers, seed=seed + 1)
    eng = vmc.Engine(sys_, prm, occ, eps=eps_opt, precision=form, cps=corr)
    vmc.Batch([eng]).autotune()
    its = O.optimize(eng, iters, sweeps, seed=seed, burn_in=burn_in, n_elec=sys_.n_elec, train_jastrow=not cps)
    J, Ca, Cb = (x.detach().cpu().numpy().copy() for x in (eng.J, eng.Ca, eng.Cb))
    opt = S.Params(J, Ca, Cb)
    corr_opt = None
    if cps:
        c = eng.c.detach().cpu().numpy()
        vals, o = [], 0
        for st in corr.sites:
            vals.append(c[o:o + 4 ** len(st)].copy())
            o += 4 ** len(st)
        corr_opt = S.CPS(corr.sites, vals)
    eng.close()
    rows = []
    for eps in eps_eval:
        ev = vmc.Engine(sys_, opt, occ, eps=eps, precision=form, cps=corr_opt)
        vmc.Batch([ev]).autotune()
        e, err, ms = sample_energy(ev, eps, eval_sweeps, 16, seed + 99)
        ns, nd, no = vmc.vmc_lists_info(ev.lists)
        rows.append({"eps_eval": eps, "energy_per_electron": e / sys_.n_elec, "error": err / sys_.n_elec,
                     "ms_per_1000_samples": 1000.0 * ms / walkers, "lists": {"singles": ns, "same": nd, "opposite": no}})
        ev.close()
        del ev
        torch.cuda.empty_cache()
    ref = rows[-1]
    for r in rows:
        r["minus_tightest_mEh_per_electron"] = 1e3 * (r["energy_per_electron"] - ref["energy_per_electron"])
        r["difference_error_mEh_per_electron"] = 1e3 * math.hypot(r["error"], ref["error"])
    return {"study": "eps_protocol", "system": name, "eps_opt": eps_opt, "walkers": walkers,
            "wavefunction": ("5-site correlators x Slater" if cps else "pair Jastrow x Slater") + f", {start} start",
            "sweeps_per_iteration": sweeps, "burn_in": burn_in, "iterations": iters,
            "form": "mixed" if form == vmc.VMC_MIXED else "fp64",
            "optimisation_last_energy_per_electron": its[-1].energy_per_electron,
            "evaluation_sweeps": eval_sweeps, "blocking": "blocks of 8 sweeps", "rows": rows}


def chain_optimisation(names=("H20", "H40", "H80", "H160"), walkers: int = 4096, sweeps: int = 64,
                       burn_in: int = 4, iters: int = 40, eps: float = 1e-6, seed: int = S.MASTER_SEED,
                       alpha0: float = 0.001, alpha1: float = 0.01, warm: int = 5,
                       form: int = vmc.VMC_MIXED, cps: bool = False, start: str = "core") -> dict:
    """The same optimisation (samples per iteration, schedule) for every chain length.  cps: the
    wavefunction is 5-site correlators x Slater determinants (the pair Jastrow set to zero and kept
    fixed), as in the paper's chain runs; start: the starting determinant (systems.make_params)."""
    out = {"study": "chain_optimisation", "walkers": walkers, "sweeps_per_iteration": sweeps, "burn_in": burn_in,
           "samples_per_iteration": walkers * (sweeps - burn_in), "eps": eps,
           "alpha": {"first": alpha0, "then": alpha1, "after_iterations": warm},
           "form": "mixed" if form == vmc.VMC_MIXED else "fp64",
           "wavefunction": ("5-site correlators x Slater" if cps else "pair Jastrow x Slater") + f", {start} start",
           "systems": {}}
    for name in names:
        sys_ = S.named_system(name)
        prm = S.make_params(sys_, seed=seed, start=start, c_noise=0.01 if start == "core" else 0.05)
        corr = None
        if cps:
            prm.J[:] = 0.0
            corr = S.make_cps(sys_, seed=seed + 7, noise=0.0)
        occ = S.init_occupations(sys_, prm, walkers, seed=seed + 1)
        eng = vmc.Engine(sys_, prm, occ, eps=eps, precision=form, cps=corr)
        vmc.Batch([eng]).autotune()
        t0 = time.perf_counter()
        its = O.optimize(eng, iters, sweeps, seed=seed, burn_in=burn_in, n_elec=sys_.n_elec, alpha0=alpha0,
                         alpha1=alpha1, warm=warm, train_jastrow=not cps)
        out["systems"][name] = {"n_params": eng.n_params, "energy_per_electron": [it.energy_per_electron for it in its],
                                "t_sum": [it.t_sum for it in its], "ms_per_iteration": float(np.median([it.ms for it in its])),
                                "rate_overflow_iterations": [it.index for it in its if it.rate_overflow],
                                "wall_s": time.perf_counter() - t0}
        eng.close()
        del eng
        torch.cuda.empty_cache()
    return out


def main():
    import argparse
    ap = argparse.ArgumentParser(description="The eps protocol (Table II) and chain-length optimisation (Fig. 2) studies")
    ap.add_argument("study", choices=["eps", "chains"])
    ap.add_argument("--systems", default="")
    ap.add_argument("--walkers", type=int, default=0)
    ap.add_argument("--sweeps", type=int, default=64)
    ap.add_argument("--iters", type=int, default=40)
    ap.add_argument("--out", default="")
    ap.add_argument("--eps", type=float, default=0.0, help="chains: screening threshold (0: 1e-6)")
    ap.add_argument("--cps", action="store_true", help="chains: 5-site correlators x Slater")
    ap.add_argument("--start", default="core", choices=["core", "neel"])
    ap.add_argument("--form", default="mixed", choices=["mixed", "fp64"])
    args = ap.parse_args()
    if args.study == "eps":
        res = [eps_protocol(n, walkers=args.walkers or 2048, sweeps=args.sweeps, iters=args.iters, cps=args.cps,
                            start=args.start, form=vmc.VMC_FP64 if args.form == "fp64" else vmc.VMC_MIXED)
               for n in (args.systems or "H20,H40").split(",")]
    else:
        res = chain_optimisation(tuple((args.systems or "H20,H40,H80,H160").split(",")), walkers=args.walkers or 4096,
                                 sweeps=args.sweeps, iters=args.iters, eps=args.eps or 1e-6, cps=args.cps,
                                 start=args.start, form=vmc.VMC_FP64 if args.form == "fp64" else vmc.VMC_MIXED)
    text = json.dumps(res)
    print(text, flush=True)
    if args.out:
        with open(args.out, "w") as f:
            f.write(text)


if __name__ == "__main__":
    main()
