#!/usr/bin/env python
"""Benchmark of the screened orbital-space VMC hot path on one GB300.

Metric: walker local-energy evaluations per second.  Workload (default): linear H160 chain,
STO-3G, 1.8 bohr, Loewdin orbitals, 80 alpha + 80 beta electrons, eps = 1e-6, 32768 walkers,
pair-Jastrow x unrestricted Slater (seeded random init, ~1e5 parameters).

One timed step = one optimisation iteration of the method: `sweeps` CTMC sweeps, each
  local energy (Eq. eloc:hci) + gradient accumulation (Eq. grad pieces) + CTMC move (Sec. II.B),
then the energy gradient, one AMSGrad update (Eqs. m1-m2) and the FP64 recompute of every
walker's tables for the new parameters (Sec. III.B).  value = walkers * sweeps / step time.

The mixed-precision form gives `value`; the FP64 form is measured the same way and reported
under "fp64_form".  `--impl reference` times the FP64 CPU oracle instead (a bounded sample).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

from paper_1807_10633_gb300 import systems as S  # noqa: E402

METRIC = "walker local-energy evals/s on 1 GB300 (H160), mixed vs FP64 form; % roofline"
UNIT = "walker-evals/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--system", default="H160")
    ap.add_argument("--walkers", type=int, default=32768)
    ap.add_argument("--sweeps", type=int, default=8, help="CTMC sweeps per optimisation iteration")
    ap.add_argument("--eps", type=float, default=1e-6)
    ap.add_argument("--forms", default="mixed,fp64")
    ap.add_argument("--cpu-sample", type=int, default=0, help="walkers in the oracle sample (0: auto)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--seed", type=int, default=S.MASTER_SEED)
    ap.add_argument("--no-graph", action="store_true", help="launch the step eagerly instead of replaying a CUDA graph")
    ap.add_argument("--no-batch", action="store_true", help="skip the uneven batched workload")
    ap.add_argument("--g-cuda-cores", action="store_true", help="form G on CUDA cores instead of tcgen05")
    ap.add_argument("--batch-walkers", type=int, default=2048)
    return ap.parse_args()


def load_system(name: str):
    cache = Path(tempfile.gettempdir()) / f"vmc_inputs_{name}.npz"
    if cache.exists():
        z = np.load(cache, allow_pickle=False)
        return S.System(name, int(z["M"]), int(z["na"]), int(z["nb"]), z["h1"], z["eri"], float(z["e_core"]))
    sys_ = S.named_system(name)
    try:
        np.savez(cache, M=sys_.M, na=sys_.n_alpha, nb=sys_.n_beta, h1=sys_.h1, eri=sys_.eri, e_core=sys_.e_core)
    except OSError:
        pass
    return sys_


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = Path(tempfile.gettempdir()) / f"vmc_clocks_{os.getpid()}.csv"

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.path.read_text().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names[1:], parts[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        self.path.unlink(missing_ok=True)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------------- our arm
def run_form(args, sys_, prm, occ, precision, rank, world, s_cnt):
    import torch
    from paper_1807_10633_gb300 import vmc

    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)               # every library call of the step runs here
    stream.wait_stream(torch.cuda.current_stream(dev))
    torch.cuda.set_stream(stream)
    eng = vmc.Engine(sys_, prm, occ, eps=args.eps, precision=precision, device=0, stream=stream)
    if args.g_cuda_cores:
        vmc.vmc_set_option(eng.ctx, vmc.VMC_OPT_G_TENSOR_CORES, 0)
    W, N2, M = eng.W, 2 * sys_.M, sys_.M
    n_singles, n_same, n_opp = vmc.vmc_lists_info(eng.lists)
    eloc_threads = vmc.Batch([eng]).autotune()    # threads per walker CTA for the local energy
    np_ = eng.n_params
    f64 = dict(dtype=torch.float64, device=dev)
    AO = torch.zeros(np_, **f64)
    AEO = torch.zeros(np_, **f64)
    g = torch.zeros(np_, **f64)
    m1 = torch.zeros(np_, **f64)
    m2 = torch.zeros(np_, **f64)
    sums = torch.zeros(2, **f64)
    AOv, AEOv = eng.split(AO), eng.split(AEO)
    ws = eng.walkers.struct()
    prm_s = eng.params
    # host buffers for the end-to-end variant (pinned)
    p_host = torch.empty(np_, dtype=torch.float64).pin_memory()
    p_host.copy_(eng.p.cpu())
    out_host = torch.empty(np_ + 2, dtype=torch.float64).pin_memory()
    ev_pairs = []   # (start, end) events around vmc_local_energy
    seed = args.seed

    def step(timed: bool, e2e: bool, it: int):
        if e2e:
            eng.p.copy_(p_host, non_blocking=True)
        AO.zero_(); AEO.zero_(); sums.zero_()
        for s in range(args.sweeps):
            if timed:
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
            vmc.vmc_local_energy(eng.ctx, eng.lists, prm_s, ws, args.eps, eng.e_loc, eng.t_res)
            if timed:
                b.record(stream)
                ev_pairs.append((a, b))
            vmc.vmc_accumulate_gradient(eng.ctx, ws, eng.t_res, eng.e_loc, AOv, AEOv, sums)
            vmc.vmc_ctmc_step(eng.ctx, eng.lists, prm_s, ws, seed + it, eng.moves)
        vmc.vmc_energy_gradient(eng.ctx, sums, AO, AEO, g)
        vmc.vmc_amsgrad_update(eng.ctx, eng.p, g, m1, m2, 0.001, 0.1, 0.01)
        vmc.vmc_walkers_refresh(eng.ctx, eng.lists, prm_s, ws)
        if e2e:
            out_host[:np_].copy_(eng.p, non_blocking=True)
            out_host[np_:].copy_(sums, non_blocking=True)
            stream.synchronize()                 # the host needs the result before its next step
            p_host.copy_(out_host[:np_])

    graph = None
    graph_launches = 0
    if not args.no_graph:
        l0 = vmc.vmc_launch_count(eng.ctx)
        step(timed=False, e2e=False, it=0)        # every workspace exists before capture
        stream.synchronize()
        graph = torch.cuda.CUDAGraph()
        l1 = vmc.vmc_launch_count(eng.ctx)
        with torch.cuda.graph(graph, stream=stream):
            step(timed=False, e2e=False, it=0)
        graph_launches = vmc.vmc_launch_count(eng.ctx) - l1      # kernels in one captured step
        del l0

    def run_step(timed: bool, e2e: bool, it: int):
        if graph is None or timed:
            step(timed=timed, e2e=e2e, it=it)
            return
        if e2e:
            eng.p.copy_(p_host, non_blocking=True)
        graph.replay()
        if e2e:
            out_host[:np_].copy_(eng.p, non_blocking=True)
            out_host[np_:].copy_(sums, non_blocking=True)
            stream.synchronize()
            p_host.copy_(out_host[:np_])

    def timed_loop(e2e: bool, it0: int):
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        launches0 = vmc.vmc_launch_count(eng.ctx)
        t0.record(stream)
        for it in range(args.steps):
            run_step(timed=False, e2e=e2e, it=it0 + it)
        t1.record(stream)
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1)
        if world > 1:
            import torch.distributed as dist
            tt = torch.tensor([ms], device=dev)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            dist.barrier()
            ms = float(tt.item())
        launches = vmc.vmc_launch_count(eng.ctx) - launches0
        if graph is not None:
            launches = graph_launches * args.steps
        return ms, launches

    for it in range(args.warmup):
        run_step(timed=False, e2e=False, it=it)
    vmc.vmc_sync(eng.ctx)
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", 0)))
    clocks.start()
    ms, launches = timed_loop(e2e=False, it0=1000)
    clk = clocks.stop()
    vmc.vmc_sync(eng.ctx)
    # local-energy launch time: CUDA events around each launch of one eager step
    torch.cuda.synchronize()
    for it in range(2):
        step(timed=True, e2e=False, it=3000 + it)
    torch.cuda.synchronize()
    vmc.vmc_sync(eng.ctx)
    eloc_ms = statistics.mean(a.elapsed_time(b) for a, b in ev_pairs)
    ms_e2e, _ = timed_loop(e2e=True, it0=2000)
    vmc.vmc_sync(eng.ctx)
    energy = float(sums[1].item() / sums[0].item())

    # algorithmic HBM bytes of one local-energy launch (walker state that must be read/written)
    esz = 8 if precision == vmc.VMC_FP64 else 4
    na, nb = sys_.n_alpha, sys_.n_beta
    ne = na + nb
    ng = (ne + 31) // 32 + sum((ne - 1 - x + 31) // 32 for x in range(ne - 1))
    occ_now = eng.walkers.occ_list.view(torch.int16).cpu().numpy().astype(np.int64).reshape(W, ne)
    f_read = 8.0 * float(np.mean(s_cnt[occ_now].sum(axis=1)))   # F entries of occupied singles
    per_walker = (esz * ((M - na) * na + (M - nb) * nb + N2)   # G virtual rows + Jastrow sums
                  + 2 * (2 * M) + 4 * 2 * ((M + 31) // 32)        # occupied / virtual lists, bits
                  + f_read + 8                                    # Fock sums of occupied singles, e_diag
                  + 16 + 16 * ng)                                 # E_L, t, rate-group sums written
    bytes_launch = per_walker * W
    achieved = bytes_launch / (eloc_ms * 1e-3) / 1e9
    evals = W * args.sweeps * args.steps
    res = dict(value=evals / (ms * 1e-3), ms_per_step=ms / args.steps, ms_e2e=ms_e2e / args.steps,
               e2e_value=evals / (ms_e2e * 1e-3), eloc_ms=eloc_ms, eloc_bytes=bytes_launch,
               eloc_gbs=achieved, launches=launches, clocks=clk, energy=energy,
               lists=dict(singles=n_singles, same=n_same, opposite=n_opp), n_params=np_, eloc_threads=eloc_threads,
               h2d=np_ * 8, d2h=(np_ + 2) * 8)
    del graph
    eng.close()
    del eng
    torch.cuda.set_stream(torch.cuda.default_stream(dev))
    torch.cuda.empty_cache()
    return res


BATCH_SYSTEMS = [("hubbard4x4", 0.0), ("hubbard6x6", 0.0), ("hubbard8x8", 0.0), ("hubbard10x10", 0.0),
                 ("H40", 1e-6), ("H60", 1e-6), ("H100", 1e-6)]


def run_batch(args):
    """Uneven batch: Hubbard L x L (U/t = 4, half filling) and H chains, one launch per sweep step."""
    import torch
    from paper_1807_10633_gb300 import vmc

    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    stream.wait_stream(torch.cuda.current_stream(dev))
    torch.cuda.set_stream(stream)
    engines = []
    for name, eps in BATCH_SYSTEMS:
        sys_ = load_system(name)
        prm = S.make_params(sys_, seed=args.seed)
        occ = S.init_occupations(sys_, prm, args.batch_walkers, seed=args.seed + 1)
        engines.append(vmc.Engine(sys_, prm, occ, eps=eps, precision=vmc.VMC_MIXED, device=0, stream=stream))
    b = vmc.Batch(engines)
    threads = b.autotune()
    f64 = dict(dtype=torch.float64, device=dev)
    acc = []
    for e in engines:
        AO, AEO = torch.zeros(e.n_params, **f64), torch.zeros(e.n_params, **f64)
        acc.append((e.split(AO), e.split(AEO), torch.zeros(2, **f64)))

    def sweep():
        b.local_energy()
        for e, (ao, aeo, sm) in zip(engines, acc):
            vmc.vmc_accumulate_gradient(e.ctx, e.walkers.struct(), e.t_res, e.e_loc, ao, aeo, sm)
        b.ctmc_step(args.seed)

    for _ in range(max(3, args.warmup)):
        sweep()
    stream.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        sweep()
    g.replay()
    stream.synchronize()
    n_sweeps = 8 * max(1, args.steps)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(n_sweeps):
        g.replay()
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / n_sweeps
    for e in engines:
        e.sync()
    res = {"systems": [n for n, _ in BATCH_SYSTEMS], "walkers_per_system": args.batch_walkers,
           "value": b.W / (ms * 1e-3), "unit": "walker-evals/s", "ms_per_sweep": ms,
           "sweep": "batched local energy + per-system gradient accumulation + batched CTMC, one CUDA graph",
           "autotuned_threads_per_walker_cta": threads, "dtype": "f32"}
    del g
    for e in engines:
        e.close()
    torch.cuda.set_stream(torch.cuda.default_stream(dev))
    torch.cuda.empty_cache()
    return res


def singles_counts(sys_, eps):
    """Length of every spatial singles list at eps (used for the byte count only)."""
    e = sys_.eri
    Jt = np.einsum("iakk->iak", e)
    Kt = np.einsum("ikka->iak", e)
    Sia = np.abs(sys_.h1) + np.abs(Jt - Kt).sum(-1) + np.abs(Jt).sum(-1)
    np.fill_diagonal(Sia, 0.0)
    cnt = (Sia > eps).sum(axis=1)
    return cnt


def cpu_sample_default() -> int:
    """Walkers in the oracle sample: 8 per host core (at most 16 cores), about 10-20 s at H160."""
    return 8 * max(1, min(os.cpu_count() or 1, 16))


def cpu_baseline(args, sys_, prm, occ, sample: int):
    import oracle
    nt = os.cpu_count() or 1
    orc = oracle.Oracle(sys_, prm)
    n = np.ascontiguousarray(oracle.occ_lists_to_n(occ[:sample], sys_.M, sys_.n_alpha))
    ctr = np.zeros(sample, dtype=np.uint64)
    t = time.perf_counter()
    orc.sweep(n, args.eps, args.seed, ctr, n_threads=nt)
    dt = time.perf_counter() - t
    return dict(value=sample / dt, unit=UNIT, cores=nt, kind="oracle",
                sample=f"{sample} walkers x 1 CTMC step (E_L + choice + move) of the same workload, "
                       f"FP64 oracle, OpenMP over walkers, {dt:.1f} s")


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    config = {"workload": f"{args.system} chain STO-3G 1.8 bohr Loewdin, eps={args.eps:g}, "
                          f"{args.walkers} walkers/GPU, {args.sweeps} CTMC sweeps per optimisation step",
              "walkers_per_gpu": args.walkers, "sweeps_per_step": args.sweeps, "eps": args.eps,
              "l2": "inputs larger than L2 (walker state > 1 GB)",
              "launch": "eager" if args.no_graph else "one CUDA graph per optimisation step"}

    sys_ = load_system(args.system)
    prm = S.make_params(sys_, seed=args.seed)
    occ = S.init_occupations(sys_, prm, args.walkers, seed=args.seed + 1)
    s_cnt = singles_counts(sys_, args.eps)

    if args.impl == "reference":
        if rank != 0:
            return
        sample = args.cpu_sample or cpu_sample_default()
        vals = []
        for _ in range(args.steps):
            vals.append(cpu_baseline(args, sys_, prm, occ, sample))
        v = statistics.median(x["value"] for x in vals)
        cb = dict(vals[0])
        cb["value"] = v
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sample / v,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": config, "cpu_baseline": cb,
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    import torch
    from paper_1807_10633_gb300 import vmc
    vmc.lib()
    forms = [f.strip() for f in args.forms.split(",") if f.strip()]
    results = {}
    for f in forms:
        results[f] = run_form(args, sys_, prm, occ, vmc.VMC_MIXED if f == "mixed" else vmc.VMC_FP64, rank, world,
                              s_cnt)
    head = results.get("mixed") or results[forms[0]]
    peak, peak_kind = measured_peaks()
    scale = world
    line = {"metric": METRIC, "value": head["value"] * scale, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if "mixed" in results else "f64", "data": "synthetic", "config": config,
            "e2e": {"value": head["e2e_value"] * scale, "unit": UNIT, "h2d_bytes_per_step": head["h2d"],
                    "d2h_bytes_per_step": head["d2h"]},
            "gpu_launches": head["launches"],
            "eloc_threads_per_walker_cta": head["eloc_threads"],
            "roofline": {"kernel": "k_local_energy", "bound": "hbm", "achieved": head["eloc_gbs"],
                         "peak": peak, "unit": "GB/s", "frac": head["eloc_gbs"] / peak,
                         "peak_source": peak_kind, "traffic": None,
                         "bytes_per_launch": head["eloc_bytes"], "launch_ms": head["eloc_ms"]},
            "clocks": head["clocks"],
            "energy_per_electron": head["energy"] / sys_.n_elec,
            "lists": head["lists"], "n_params": head["n_params"]}
    for f, r in results.items():
        if f != "mixed" or len(results) == 1:
            line[f"{f}_form"] = {"value": r["value"] * scale, "ms_per_step": r["ms_per_step"],
                                 "eloc_ms": r["eloc_ms"], "eloc_gbs": r["eloc_gbs"],
                                 "e2e_value": r["e2e_value"] * scale, "energy_per_electron": r["energy"] / sys_.n_elec}
    if "mixed" in results and "fp64" in results:
        line["mixed_over_fp64"] = results["mixed"]["value"] / results["fp64"]["value"]
    if not args.no_batch:
        line["batched_uneven"] = run_batch(args)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sample = args.cpu_sample or cpu_sample_default()
        line["cpu_baseline"] = cpu_baseline(args, sys_, prm, occ, sample)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
