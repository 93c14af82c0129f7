"""Writes tests/golden/oracle_regression.json: outputs of the oracle (and only the oracle) on
small seeded workloads, so that a later change to the oracle that moves its results is seen.
These are regression values, not pins: the pins that tie the oracle to the paper and to the
mathematics are in tests/test_oracle_pins.py and tests/test_oracle_cps.py.

    python tests/golden/make_oracle_regression.py
"""
import json
import sys
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

import oracle  # noqa: E402
from paper_1807_10633_gb300 import systems as S  # noqa: E402

CASES = [("hubbard10", 0.0, 32, 3), ("H20", 1e-6, 8, 2)]   # (system, eps, walkers, CTMC steps)
SEED = 2718


def run_case(name, eps, W, steps):
    sys_ = S.named_system(name)
    prm = S.make_params(sys_, seed=S.MASTER_SEED)
    occ = S.init_occupations(sys_, prm, W, seed=S.MASTER_SEED + 1)
    n = np.ascontiguousarray(oracle.occ_lists_to_n(occ, sys_.M, sys_.n_alpha))
    orc = oracle.Oracle(sys_, prm)
    ctr = np.zeros(W, dtype=np.uint64)
    out = {"e_loc": [], "t_res": [], "moves": []}
    for _ in range(steps):
        el, tr, mv, err = orc.sweep(n, eps, SEED, ctr, n_threads=1)
        assert err == 0
        out["e_loc"].append(el.tolist())
        out["t_res"].append(tr.tolist())
        out["moves"].append(mv.tolist())
    out["final_occupations"] = n.astype(int).tolist()
    return out


def main():
    data = {"_note": "oracle outputs (regression values); written by tests/golden/make_oracle_regression.py",
            "seed": SEED, "cases": {}}
    for name, eps, W, steps in CASES:
        data["cases"][name] = dict(eps=eps, walkers=W, steps=steps, **run_case(name, eps, W, steps))
    (Path(__file__).parent / "oracle_regression.json").write_text(json.dumps(data))


if __name__ == "__main__":
    main()
