#!/usr/bin/env python
"""Benchmark of the screened orbital-space VMC hot path on one GB300.

Metric: walker local-energy evaluations per second.  Workload (default): linear H160 chain,
STO-3G, 1.8 bohr, Loewdin orbitals, 80 alpha + 80 beta electrons, eps = 1e-6, 32768 walkers,
pair-Jastrow x unrestricted Slater (seeded random init, ~1e5 parameters).

One timed step = one optimisation iteration of the method: `sweeps` CTMC sweeps, each
  local energy (Eq. eloc:hci) + gradient accumulation (Eq. grad pieces) + CTMC move (Sec. II.B),
then the energy gradient, one AMSGrad update (Eqs. m1-m2) and the FP64 recompute of every
walker's tables for the new parameters (Sec. III.B).  value = walkers * sweeps / step time.

The mixed-precision form gives `value` (FP32 tables and ratios, C_occ factorised by FP64 LU at each
refresh, G on the tensor cores); the FP64 form ("fp64_form") and the mixed form with an FP32
Gauss-Jordan refresh ("mixed_gj32_form") are measured the same way.  `--impl reference` times
the FP64 CPU oracle instead (a bounded sample).

Under torchrun (N > 1) every rank runs its own walkers and the walker sums are added by one
all-reduce per step (NCCL; VMC_DIST_BACKEND=gloo uses gloo, which also lets ranks share a GPU);
the line reports `replicas_identical`, whether every rank's parameters equal rank 0's at the end.
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
    ap.add_argument("--forms", default="mixed,fp64,mixed_gj32,mixed_cps",
                    help="mixed: FP32 tables, FP64 LU of C_occ at every refresh; fp64: FP64 throughout; "
                         "mixed_gj32: FP32 tables, FP32 Gauss-Jordan refresh; mixed_cps: the mixed form with "
                         "5-site correlators on every site multiplying the wavefunction (Sec. III.A)")
    ap.add_argument("--cpu-sample", type=int, default=0, help="walkers in the oracle sample (0: auto)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--seed", type=int, default=S.MASTER_SEED)
    ap.add_argument("--no-graph", action="store_true", help="launch the step eagerly instead of replaying a CUDA graph")
    ap.add_argument("--no-batch", action="store_true", help="skip the uneven batched workload")
    ap.add_argument("--g-cuda-cores", action="store_true", help="form G on CUDA cores instead of tcgen05")
    ap.add_argument("--grad-j-int", action="store_true",
                    help="sum the Jastrow gradient block on the integer pipe instead of tcgen05")
    ap.add_argument("--batch-walkers", type=int, default=2048)
    ap.add_argument("--eps-sweep", default="", help="comma-separated eps values: run the eps / size study "
                    "(cost per 1000 samples of H chains) instead of the benchmark")
    ap.add_argument("--study-systems", default="H20,H40,H80,H160")
    ap.add_argument("--repeats", type=int, default=2,
                    help="pairs of timed loops of K steps (device-timed and end to end); medians are reported")
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


def l2_note(system: str, walkers: int) -> str:
    """Whether the walker tables (G and C_occ^-1 per spin, FP32 in the mixed form) exceed the 129 MB
    L2, so that every sweep streams them from HBM without an L2 flush between steps."""
    sys_ = S.named_system(system) if system.startswith("hubbard") else None
    if sys_ is None:
        M = int(system[1:]) if system.startswith("H") else 0
        na = nb = M // 2
    else:
        M, na, nb = sys_.M, sys_.n_alpha, sys_.n_beta
    tables = 4 * walkers * ((M - na) * na + (M - nb) * nb + na * na + nb * nb)
    if tables > 129e6:
        return f"inputs larger than L2 (walker tables {tables / 1e9:.2f} GB in FP32, no flush needed)"
    return f"walker tables fit in L2 ({tables / 1e6:.1f} MB in FP32): a small case, not a timing configuration"


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


# ncu counters of one k_local_energy launch (mixed form, H160, eps 1e-6, 4,096 walkers), per walker:
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum), L2 bytes (lts__t_sectors.sum x 32) and
# warp instructions (smsp__inst_executed.sum), from the capture summarised in
# profiles/k_local_energy_mixed_h160_w4096.md.  They describe the kernel source with this digest
# only; any later change of the kernel's file reports traffic as null until it is captured again.
ELOC_COUNTERS = {"sha256": "2ce2119c06f96ce3069d3b8429e711f38fb44c503e99b0be541f82c9f7cb0725",
                 "system": "H160", "eps": 1e-6, "dram_bytes_per_walker": 80584.9, "l2_bytes_per_walker": 875568.0,
                 "warp_inst_per_walker": 219949.0}


def counters_apply(system: str, eps: float) -> bool:
    """The captured counters describe this workload and the kernel source as it is now."""
    return (eloc_source_digest() == ELOC_COUNTERS["sha256"] and system == ELOC_COUNTERS["system"]
            and eps == ELOC_COUNTERS["eps"])


def eloc_source_digest() -> str:
    import hashlib
    h = hashlib.sha256()
    h.update((ROOT / "paper_1807_10633_gb300" / "csrc" / "eloc.cu").read_bytes())
    return h.hexdigest()


def l2_probe_gbs(dev) -> float:
    """L2 read bandwidth: the library's read-only probe kernel over a 48 MB buffer that stays in the
    129 MB L2 (16-byte loads through L2, bypassing L1), best of five timed launches of 20 passes."""
    import torch
    from paper_1807_10633_gb300 import vmc
    buf = torch.ones(48 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    ctx = vmc.vmc_create(dev.index, stream)
    try:
        vmc.vmc_probe_l2_read(ctx, buf, 2)                 # brings the buffer into L2
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        best = None
        for _ in range(5):
            t0.record(stream)
            vmc.vmc_probe_l2_read(ctx, buf, 20)
            t1.record(stream)
            torch.cuda.synchronize()
            ms = t0.elapsed_time(t1)
            best = ms if best is None else min(best, ms)
    finally:
        vmc.vmc_destroy(ctx)
    return 20 * buf.numel() * 4 / (best * 1e-3) / 1e9


def measured_peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------------- our arm
RATE_OVERFLOW = 6      # VMC_ERR_OVERFLOW


def sync_counting_overflow(vmc, eng) -> bool:
    """Wait for the engine's stream; a CTMC rate clamped at the fixed-point limit (a walker on a
    near-node determinant of the wavefunction the step keeps optimising; its weight is nil) is
    reported, not fatal.  Any other latched error is raised."""
    st = vmc.lib().vmc_sync(eng.ctx)
    if st not in (0, RATE_OVERFLOW):
        vmc._check(eng.ctx, st)
    return st == RATE_OVERFLOW


def run_form(args, sys_, prm, occ, precision, rank, world, gj32=False, cps=None):
    import torch
    from paper_1807_10633_gb300 import vmc

    from paper_1807_10633_gb300 import dist as D

    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream(dev)               # every library call of the step runs here
    stream.wait_stream(torch.cuda.current_stream(dev))
    torch.cuda.set_stream(stream)
    eng = vmc.Engine(sys_, prm, occ, eps=args.eps, precision=precision, device=dev.index, stream=stream, cps=cps)
    if args.g_cuda_cores:
        vmc.vmc_set_option(eng.ctx, vmc.VMC_OPT_G_TENSOR_CORES, 0)
    if args.grad_j_int:
        vmc.vmc_set_option(eng.ctx, vmc.VMC_OPT_GRAD_J_TENSOR_CORES, 0)
    if gj32:   # mixed tables, C_occ inverted by FP32 Gauss-Jordan at every refresh
        vmc.vmc_set_option(eng.ctx, vmc.VMC_OPT_MIXED_REFRESH_GJ32, 1)
        eng.refresh()
    W, N2, M = eng.W, 2 * sys_.M, sys_.M
    n_singles, n_same, n_opp = vmc.vmc_lists_info(eng.lists)
    eloc_threads = vmc.Batch([eng]).autotune()    # threads per walker CTA for the local energy
    e_start, _ = eng.local_energy()               # every form starts from the same determinants
    e_start = e_start.cpu().numpy().copy()
    np_ = eng.n_params
    f64 = dict(dtype=torch.float64, device=dev)
    red, AO, AEO, sums = D.sums_buffer(np_, dev)   # the walker sums: one buffer, one exchange
    g = torch.zeros(np_, **f64)
    m1 = torch.zeros(np_, **f64)
    m2 = torch.zeros(np_, **f64)
    AOv, AEOv = eng.split(AO), eng.split(AEO)
    AOc, AEOc = eng.split_cps(AO), eng.split_cps(AEO)     # correlator coefficients (None without them)
    ws = eng.walkers.struct()
    prm_s = eng.params
    # host buffers for the end-to-end variant (pinned)
    p_host = torch.empty(np_, dtype=torch.float64).pin_memory()
    p_host.copy_(eng.p.cpu())
    out_host = torch.empty(np_ + 2, dtype=torch.float64).pin_memory()
    ev_pairs = []   # (start, end) events around vmc_local_energy
    seed = args.seed

    def sweeps(timed: bool, it: int):
        red.zero_()
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
            if AOc is not None:
                vmc.vmc_accumulate_gradient_cps(eng.ctx, ws, prm_s, eng.t_res, eng.e_loc, AOc, AEOc)
            vmc.vmc_ctmc_step(eng.ctx, eng.lists, prm_s, ws, D.rank_seed(seed + it, rank), eng.moves)

    def update():
        vmc.vmc_energy_gradient(eng.ctx, sums, AO, AEO, g)
        vmc.vmc_amsgrad_update(eng.ctx, eng.p, g, m1, m2, 0.001, 0.1, 0.01)
        vmc.vmc_walkers_refresh(eng.ctx, eng.lists, prm_s, ws)

    def step(timed: bool, e2e: bool, it: int):
        if e2e:
            eng.p.copy_(p_host, non_blocking=True)
        sweeps(timed, it)
        D.allreduce_sums(red)                    # N > 1: the one exchange of the iteration
        update()
        if e2e:
            out_host[:np_].copy_(eng.p, non_blocking=True)
            out_host[np_:].copy_(sums, non_blocking=True)
            stream.synchronize()                 # the host needs the result before its next step
            p_host.copy_(out_host[:np_])

    graph = None          # one graph per step (N = 1), or sweeps and update around the exchange
    graph_b = None
    graph_launches = 0
    if not args.no_graph:
        step(timed=False, e2e=False, it=0)        # every workspace exists before capture
        stream.synchronize()
        graph = torch.cuda.CUDAGraph()
        l1 = vmc.vmc_launch_count(eng.ctx)
        if world == 1:
            with torch.cuda.graph(graph, stream=stream):
                step(timed=False, e2e=False, it=0)
        else:
            with torch.cuda.graph(graph, stream=stream):
                sweeps(False, 0)
            graph_b = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph_b, stream=stream):
                update()
        graph_launches = vmc.vmc_launch_count(eng.ctx) - l1      # kernels in one captured step

    def run_step(timed: bool, e2e: bool, it: int):
        if graph is None or timed:
            step(timed=timed, e2e=e2e, it=it)
            return
        if e2e:
            eng.p.copy_(p_host, non_blocking=True)
        graph.replay()
        if graph_b is not None:
            D.allreduce_sums(red)
            graph_b.replay()
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

    overflow = False
    for it in range(args.warmup):
        run_step(timed=False, e2e=False, it=it)
    overflow |= sync_counting_overflow(vmc, eng)
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    dev_ms, e2e_ms = [], []
    # device-timed and end-to-end loops in the order d e | e d | d e | ...: every step moves the
    # parameters, so the workload drifts slowly; this order gives both arms the same mean position
    for r in range(args.repeats):
        for k, e2e in enumerate((False, True) if r % 2 == 0 else (True, False)):
            ms_r, launches_r = timed_loop(e2e=e2e, it0=1000 + (2 * r + k) * args.steps)
            (e2e_ms if e2e else dev_ms).append(ms_r)
            if not e2e:
                launches = launches_r
    clk = clocks.stop()
    overflow |= sync_counting_overflow(vmc, eng)
    ms, ms_e2e = statistics.median(dev_ms), statistics.median(e2e_ms)
    # local-energy launch time: CUDA events around each launch of one eager step
    torch.cuda.synchronize()
    for it in range(2):
        step(timed=True, e2e=False, it=3000 + it)
    torch.cuda.synchronize()
    overflow |= sync_counting_overflow(vmc, eng)
    eloc_ms = statistics.mean(a.elapsed_time(b) for a, b in ev_pairs)
    energy = float(sums[1].item() / sums[0].item())

    # Algorithmic bytes of one local-energy launch, the per-eval figure of the scope table:
    #   B_eval = K_d b_d + K_s b_s + (F reads of the free singles) + B_state
    # with K_d, K_s the double and single list entries each walker's walk reads, measured by the
    # library (vmc_screened_moves) on the walkers as the timed run left them; b_d = 8 B mixed /
    # 12 B FP64 (a, b, v), b_s = 12 / 16 B; one Fock-sum element per free single (this design keeps
    # them per walker instead of re-reading O(N_e) integral rows); B_state = the walker state the
    # launch reads and writes.
    esz = 8 if precision == vmc.VMC_FP64 else 4
    na, nb = sys_.n_alpha, sys_.n_beta
    ng = eng_groups(sys_, eng)
    n_moves, walked = eng.move_counts()
    k_s, k_d = float(walked[:, 0].mean()), float(walked[:, 1].mean())
    b_d, b_s = (12, 16) if precision == vmc.VMC_FP64 else (8, 12)
    state = (esz * ((M - na) * na + (M - nb) * nb + N2)       # G virtual rows + Jastrow sums
             + 2 * (2 * M) + 8                                 # orbital map, e_diag
             + 16 + (16 + 8) * ng)                             # E_L, t; rate sums and energy partials
    free_s = float(np.mean(singles_free(eng, n_moves)))
    per_eval = k_d * b_d + k_s * b_s + free_s * esz + state
    bytes_launch = per_eval * W
    achieved = bytes_launch / (eloc_ms * 1e-3) / 1e9
    evals = W * args.sweeps * args.steps
    spread = lambda xs: (max(xs) - min(xs)) / statistics.median(xs)
    res = dict(value=evals / (ms * 1e-3), ms_per_step=ms / args.steps, ms_e2e=ms_e2e / args.steps,
               e2e_value=evals / (ms_e2e * 1e-3), eloc_ms=eloc_ms, eloc_bytes=bytes_launch,
               eloc_gbs=achieved, launches=launches, clocks=clk, energy=energy,
               repeats=dict(n=args.repeats, ms_per_step=[x / args.steps for x in dev_ms],
                            e2e_ms_per_step=[x / args.steps for x in e2e_ms],
                            spread=spread(dev_ms), e2e_spread=spread(e2e_ms)),
               per_walker=dict(K_d_walked=k_d, K_s_walked=k_s, moves=float(n_moves.mean()),
                               singles_free=free_s, b_d=b_d, b_s=b_s, state_bytes=state,
                               bytes_per_eval=per_eval, groups=ng),
               e_start=e_start, rate_overflow=overflow,
               lists=dict(singles=n_singles, same=n_same, opposite=n_opp), n_params=np_, eloc_threads=eloc_threads,
               h2d=np_ * 8, d2h=(np_ + 2) * 8)
    if world > 1:
        # the replicas of the parameters must stay identical on every rank (the same reduced
        # gradient, the same AMSGrad update): compare each rank's copy with rank 0's
        import torch.distributed as dist
        ref = eng.p.clone()
        dist.broadcast(ref, 0)
        bad = torch.tensor([0.0 if torch.equal(ref, eng.p) else 1.0], dtype=torch.float64, device=dev)
        dist.all_reduce(bad, op=dist.ReduceOp.MAX)
        res["replicas_identical"] = bool(bad.item() == 0.0)
    del graph
    eng.close()
    del eng
    torch.cuda.set_stream(torch.cuda.default_stream(dev))
    torch.cuda.empty_cache()
    return res


def eng_groups(sys_, eng) -> int:
    """Warp groups per walker of the local energy (the rate store's groups): singles blocks of 32
    spin orbitals plus the row groups of the pair band (equal to the library's count)."""
    from paper_1807_10633_gb300 import vmc
    return vmc.vmc_lists_layout(eng.lists)["n_groups"]


def singles_free(eng, n_moves):
    """Free singles per walker: moves that are singles, from one walker sample's move codes."""
    k = min(eng.W, 64)
    per, _, _ = eng.screened_moves(0, k)
    return [int(((c & 3) == 1).sum()) for c, _, _ in per]


BATCH_SYSTEMS = [("hubbard4x4", 0.0), ("hubbard6x6", 0.0), ("hubbard8x8", 0.0), ("hubbard10x10", 0.0),
                 ("H40", 1e-6), ("H60", 1e-6), ("H100", 1e-6)]


def run_batch(args):
    """Uneven batch: Hubbard L x L (U/t = 4, half filling) and H chains, one launch per sweep step."""
    import torch
    from paper_1807_10633_gb300 import vmc

    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream(dev)
    stream.wait_stream(torch.cuda.current_stream(dev))
    torch.cuda.set_stream(stream)
    engines = []
    for name, eps in BATCH_SYSTEMS:
        sys_ = load_system(name)
        prm = S.make_params(sys_, seed=args.seed)
        occ = S.init_occupations(sys_, prm, args.batch_walkers, seed=args.seed + 1)
        engines.append(vmc.Engine(sys_, prm, occ, eps=eps, precision=vmc.VMC_MIXED, device=dev.index, stream=stream))
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


def eps_study(args):
    """Cost per 1000 samples (local energy + CTMC move, mixed form) against eps and chain length,
    and the fitted exponent of cost per sample against the number of orbitals at each eps."""
    import torch
    from paper_1807_10633_gb300 import vmc

    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    eps_list = [float(e) for e in args.eps_sweep.split(",") if e.strip()]
    rows = []
    for name in [x.strip() for x in args.study_systems.split(",") if x.strip()]:
        sys_ = load_system(name)
        prm = S.make_params(sys_, seed=args.seed)
        occ = S.init_occupations(sys_, prm, args.walkers, seed=args.seed + 1)
        for eps in eps_list:
            eng = vmc.Engine(sys_, prm, occ, eps=eps, precision=vmc.VMC_MIXED, device=dev.index, stream=stream)
            vmc.Batch([eng]).autotune()
            ns, nd, no = vmc.vmc_lists_info(eng.lists)
            ws, prm_s = eng.walkers.struct(), eng.params

            def sweep(k):
                vmc.vmc_local_energy(eng.ctx, eng.lists, prm_s, ws, eps, eng.e_loc, eng.t_res)
                vmc.vmc_ctmc_step(eng.ctx, eng.lists, prm_s, ws, args.seed + k, eng.moves)
            for k in range(3):
                sweep(k)
            eng.sync()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            n_sw = max(2, args.sweeps)
            a.record(stream)
            for k in range(n_sw):
                sweep(100 + k)
            b.record(stream)
            torch.cuda.synchronize()
            eng.sync()
            ms = a.elapsed_time(b) / n_sw
            e_mean = float((eng.t_res * eng.e_loc).sum() / eng.t_res.sum())
            rows.append({"system": name, "M": sys_.M, "eps": eps, "walkers": args.walkers,
                         "lists": {"singles": ns, "same": nd, "opposite": no},
                         "ms_per_sweep": ms, "ms_per_1000_samples": 1000.0 * ms / args.walkers,
                         "energy_per_electron": e_mean / sys_.n_elec})
            print(json.dumps(rows[-1]), flush=True)
            eng.close()
            del eng
            torch.cuda.empty_cache()
    fits = {}
    for eps in eps_list:
        pts = [(r["M"], r["ms_per_1000_samples"]) for r in rows if r["eps"] == eps]
        if len(pts) >= 2:
            x = np.log([p[0] for p in pts]); y = np.log([p[1] for p in pts])
            fits[f"{eps:g}"] = float(np.polyfit(x, y, 1)[0])
    print(json.dumps({"study": "eps_and_size", "unit": "ms per 1000 samples (local energy + CTMC move)",
                      "form": "mixed", "rows": len(rows), "exponent_vs_orbitals": fits}), flush=True)


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
    el, _, _, _ = orc.sweep(n, args.eps, args.seed, ctr, n_threads=nt)
    dt = time.perf_counter() - t
    # one thread on a few of the same walkers (the oracle's single-core rate)
    s1 = max(1, min(sample, 4))
    n1 = np.ascontiguousarray(oracle.occ_lists_to_n(occ[:s1], sys_.M, sys_.n_alpha))
    t = time.perf_counter()
    orc.sweep(n1, args.eps, args.seed, np.zeros(s1, dtype=np.uint64), n_threads=1)
    dt1 = time.perf_counter() - t
    return dict(value=sample / dt, unit=UNIT, cores=nt, kind="oracle",
                sample=f"{sample} walkers x 1 CTMC step (E_L + choice + move) of the same workload, "
                       f"FP64 oracle, OpenMP over walkers, {dt:.1f} s",
                single_thread={"value": s1 / dt1, "unit": UNIT, "cores": 1,
                               "sample": f"{s1} walkers x 1 CTMC step on one thread, {dt1:.1f} s"},
                e_loc=el)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference" and rank != 0:
        return                     # the CPU reference arm runs on rank 0 alone, with no process group
    if world > 1 and args.impl != "reference":
        import torch
        import torch.distributed as dist
        # one rank per GPU; VMC_DIST_BACKEND=gloo runs the same exchange through host memory, which
        # also lets several ranks share one GPU (their kernels never wait on one another)
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)) % torch.cuda.device_count())
        dist.init_process_group(os.environ.get("VMC_DIST_BACKEND", "nccl"))
    if args.eps_sweep:
        if rank == 0:
            eps_study(args)
        return
    config = {"workload": f"{args.system} chain STO-3G 1.8 bohr Loewdin, eps={args.eps:g}, "
                          f"{args.walkers} walkers/GPU, {args.sweeps} CTMC sweeps per optimisation step",
              "walkers_per_gpu": args.walkers, "sweeps_per_step": args.sweeps, "eps": args.eps,
              "l2": l2_note(args.system, args.walkers),
              "launch": "eager" if args.no_graph else "one CUDA graph per optimisation step",
              "parallelism": (f"walkers sharded over {world} GPUs, one all-reduce of the walker sums per "
                              f"optimisation step ({os.environ.get('VMC_DIST_BACKEND', 'nccl')}), "
                              f"parameters replicated") if world > 1 else "1 GPU"}

    sys_ = load_system(args.system)
    prm = S.make_params(sys_, seed=args.seed)
    # each rank's own walkers (weak scaling: walkers per GPU fixed); rank 0 keeps the 1-GPU inputs
    occ = S.init_occupations(sys_, prm, args.walkers, seed=args.seed + 1 + 1000003 * rank)

    if args.impl == "reference":
        sample = args.cpu_sample or cpu_sample_default()
        vals = []
        for _ in range(args.steps):
            vals.append(cpu_baseline(args, sys_, prm, occ, sample))
        v = statistics.median(x["value"] for x in vals)
        cb = dict(vals[0])
        cb.pop("e_loc")
        cb["value"] = v
        config = dict(config, launch="FP64 CPU oracle, OpenMP over walkers", l2="not applicable (CPU)")
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
        cps = S.make_cps(sys_, seed=args.seed + 7, noise=0.05) if f.endswith("_cps") else None
        results[f] = run_form(args, sys_, prm, occ, vmc.VMC_FP64 if f == "fp64" else vmc.VMC_MIXED, rank, world,
                              gj32=(f == "mixed_gj32"), cps=cps)
    head = results.get("mixed") or results[forms[0]]
    peak, peak_kind = measured_peaks()
    counters_ok = "mixed" in results and counters_apply(args.system, args.eps)
    traffic = ELOC_COUNTERS["dram_bytes_per_walker"] * args.walkers if counters_ok else None
    l2_peak = l2_probe_gbs(torch.device("cuda", torch.cuda.current_device()))
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    sm_mhz = head["clocks"].get("sm_mhz") or head["clocks"].get("sm_max_mhz") or 2070.0
    issue_peak = 4 * props.multi_processor_count * sm_mhz * 1e6 / 1e12     # Twarp-inst/s
    l2_bytes = ELOC_COUNTERS["l2_bytes_per_walker"] * args.walkers if counters_ok else None
    launch_s = head["eloc_ms"] * 1e-3
    pw = head["per_walker"]
    scale = world
    line = {"metric": METRIC, "value": head["value"] * scale, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if "mixed" in results else "f64", "data": "synthetic", "config": config,
            "e2e": {"value": head["e2e_value"] * scale, "unit": UNIT, "h2d_bytes_per_step": head["h2d"],
                    "d2h_bytes_per_step": head["d2h"]},
            "repeats": head["repeats"],
            "gpu_launches": head["launches"],
            "eloc_threads_per_walker_cta": head["eloc_threads"],
            "roofline": {"kernel": "k_local_energy", "bound": "hbm", "achieved": head["eloc_gbs"],
                         "peak": peak, "unit": "GB/s", "frac": head["eloc_gbs"] / peak,
                         "peak_source": peak_kind, "traffic": traffic,
                         "bytes_per_launch": head["eloc_bytes"], "launch_ms": head["eloc_ms"],
                         "bytes": "B_eval = K_d b_d + K_s b_s + free singles x F element + walker state, "
                                  "K_d and K_s measured per walker by the library (per_walker)",
                         "per_walker": pw,
                         "state_only_frac": pw["state_bytes"] * args.walkers / launch_s / 1e9 / peak},
            "issue_roofline": {"kernel": "k_local_energy", "bound": "issue",
                               "achieved": (ELOC_COUNTERS["warp_inst_per_walker"] * args.walkers /
                                            launch_s / 1e12) if counters_ok else None,
                               "peak": issue_peak, "unit": "Twarp-inst/s",
                               "frac": (ELOC_COUNTERS["warp_inst_per_walker"] * args.walkers /
                                        launch_s / 1e12 / issue_peak) if counters_ok else None,
                               "peak_source": "4 schedulers x SMs x median SM clock under load, one warp "
                                              "instruction per scheduler per clock"},
            "l2_roofline": {"kernel": "k_local_energy", "bound": "l2",
                            "achieved": (l2_bytes / launch_s / 1e9) if l2_bytes else None,
                            "peak": l2_peak, "unit": "GB/s",
                            "frac": (l2_bytes / launch_s / 1e9 / l2_peak) if l2_bytes else None,
                            "bytes": "ncu lts__t_sectors x 32 per launch, scaled by walkers",
                            "peak_source": "the library's L2-resident read probe (vmc_probe_l2_read, 48 MB)"},
            "clocks": head["clocks"],
            "rate_overflow": {f: r["rate_overflow"] for f, r in results.items()},
            "energy_per_electron": head["energy"] / sys_.n_elec,
            "lists": head["lists"], "n_params": head["n_params"]}
    if world > 1:
        line["replicas_identical"] = all(r["replicas_identical"] for r in results.values())
    for f, r in results.items():
        if f != "mixed" or len(results) == 1:
            line[f"{f}_form"] = {"value": r["value"] * scale, "ms_per_step": r["ms_per_step"],
                                 "n_params": r["n_params"],
                                 "eloc_ms": r["eloc_ms"], "eloc_gbs": r["eloc_gbs"],
                                 "e2e_value": r["e2e_value"] * scale, "repeats": r["repeats"],
                                 "energy_per_electron": r["energy"] / sys_.n_elec}
    if "mixed" in results and "fp64" in results:
        line["mixed_over_fp64"] = results["mixed"]["value"] / results["fp64"]["value"]
    # error of the mixed forms against the FP64 form, every walker at the common start (mEh / electron)
    if "fp64" in results:
        ref = results["fp64"]["e_start"]
        line["mixed_error"] = {f: {"max_mEh_per_electron": float(np.max(np.abs(r["e_start"] - ref))) * 1e3 / sys_.n_elec,
                                   "mean_mEh_per_electron": float(np.mean(np.abs(r["e_start"] - ref))) * 1e3 / sys_.n_elec,
                                   "walkers": int(ref.size), "against": "FP64 form on the GPU, same determinants"}
                               for f, r in results.items() if f != "fp64" and not f.endswith("_cps")}
    if not args.no_batch:
        line["batched_uneven"] = run_batch(args)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sample = args.cpu_sample or cpu_sample_default()
        cb = cpu_baseline(args, sys_, prm, occ, sample)
        el_orc = cb.pop("e_loc")
        cb["parity_sample"] = {f: (float(np.max(np.abs(r["e_start"][:sample] - el_orc) / np.maximum(1.0, np.abs(el_orc))))
                                   if f == "fp64" else
                                   float(np.max(np.abs(r["e_start"][:sample] - el_orc))) * 1e3 / sys_.n_elec)
                               for f, r in results.items() if not f.endswith("_cps")}
        cb["parity_sample_units"] = "fp64: max relative E_L error; mixed forms: max mEh per electron"
        line["cpu_baseline"] = cb
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
