"""The reference arm of bench.py (the FP64 oracle on the host cores, a bounded sample) prints one
JSON line with the benchmark's keys, once, from rank 0 only; CPU only."""
import json
import os
import subprocess
import sys
from pathlib import Path

ROOT = Path(__file__).resolve().parents[1]
ARGS = ["--impl", "reference", "--system", "H20", "--walkers", "64", "--cpu-sample", "8",
        "--steps", "2", "--warmup", "3"]
KEYS = {"impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
        "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"}


def _lines(out: str):
    return [json.loads(x) for x in out.splitlines() if x.startswith("{")]


def test_reference_arm_prints_one_line_with_the_contract_keys():
    r = subprocess.run([sys.executable, str(ROOT / "bench.py"), *ARGS], cwd=ROOT, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    (line,) = _lines(r.stdout)
    assert KEYS <= set(line)
    assert line["impl"] == "reference" and line["higher_is_better"] is True and line["steps"] == 2
    assert line["value"] > 0 and line["e2e"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1 and cb["sample"]
    assert "workload" in line["config"]


def _free_port() -> int:
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_reference_arm_under_two_ranks_prints_once():
    env = dict(os.environ, MASTER_ADDR="127.0.0.1")
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
                        "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), str(ROOT / "bench.py"),
                        "--gpus", "2", *ARGS], cwd=ROOT, capture_output=True, text=True, timeout=300, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    (line,) = _lines(r.stdout)
    assert line["impl"] == "reference" and line["n_gpus"] == 2


def test_ncu_counters_are_reported_only_for_the_captured_kernel_source(monkeypatch):
    """The DRAM/L2/instruction counters bench.py reports for the local-energy kernel were taken on
    the kernel source with a recorded digest; once that file changes they no longer describe the
    kernel, and bench.py must report traffic as null until a new capture is recorded."""
    sys.path.insert(0, str(ROOT))
    import bench
    current = bench.eloc_source_digest() == bench.ELOC_COUNTERS["sha256"]
    assert bench.counters_apply("H160", 1e-6) == current
    assert not bench.counters_apply("H80", 1e-6)
    monkeypatch.setitem(bench.ELOC_COUNTERS, "sha256", bench.eloc_source_digest())
    assert bench.counters_apply("H160", 1e-6)
    monkeypatch.setitem(bench.ELOC_COUNTERS, "sha256", "0" * 64)
    assert not bench.counters_apply("H160", 1e-6)


def test_l2_note_follows_the_walker_tables():
    """The config's L2 statement: the H160 benchmark's walker tables (G and C_occ^-1 of both spins,
    FP32) are 3.36 GB, far above the 129 MB L2, so no flush is needed between timed steps; a small
    case is labelled as one."""
    sys.path.insert(0, str(ROOT))
    import bench
    big = bench.l2_note("H160", 32768)
    assert big.startswith("inputs larger than L2") and "3.36 GB" in big
    assert bench.l2_note("H20", 512).startswith("walker tables fit in L2")
