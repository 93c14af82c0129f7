"""The oracle still produces the outputs stored by tests/golden/make_oracle_regression.py (a
regression guard for changes to the oracle; the pins are elsewhere).  CPU only."""
import json
from pathlib import Path

import numpy as np
import pytest

from tests.golden import make_oracle_regression as R

GOLD = json.loads((Path(__file__).parent / "golden" / "oracle_regression.json").read_text())


@pytest.mark.parametrize("name,eps,W,steps", R.CASES, ids=[c[0] for c in R.CASES])
def test_oracle_outputs_unchanged(name, eps, W, steps):
    ref = GOLD["cases"][name]
    got = R.run_case(name, eps, W, steps)
    np.testing.assert_allclose(got["e_loc"], ref["e_loc"], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(got["t_res"], ref["t_res"], rtol=1e-12, atol=0)
    assert got["moves"] == ref["moves"]
    assert got["final_occupations"] == ref["final_occupations"]
