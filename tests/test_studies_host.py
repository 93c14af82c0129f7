"""Host logic of the studies module (CPU only): the blocking error estimate of a residence-time
weighted mean."""
import math

import numpy as np
import pytest

from paper_1807_10633_gb300.studies import blocking_error


def test_blocking_mean_is_the_weighted_mean_and_iid_error_matches_theory():
    rng = np.random.default_rng(3)
    S, W = 512, 64
    e = rng.normal(1.5, 2.0, size=(S, W))
    t = np.ones((S, W))
    E, err = blocking_error(e, t, block=8)
    assert E == pytest.approx(e.mean(), rel=1e-14)
    # independent samples: the error of the mean is sigma / sqrt(S W) whatever the block length
    assert err == pytest.approx(2.0 / math.sqrt(S * W), rel=0.2)


def test_blocking_sees_correlation_between_consecutive_sweeps():
    rng = np.random.default_rng(4)
    S, W = 1024, 16
    x = np.zeros((S, W))
    for s in range(1, S):                  # AR(1) over sweeps, correlation time ~ 20 sweeps
        x[s] = 0.95 * x[s - 1] + rng.normal(size=W)
    t = rng.uniform(0.5, 1.5, size=(S, W))
    _, e1 = blocking_error(x, t, block=1)
    _, e64 = blocking_error(x, t, block=64)
    assert e64 > 3 * e1                    # short blocks underestimate correlated errors


def test_blocking_needs_two_blocks():
    with pytest.raises(ValueError):
        blocking_error(np.zeros((8, 2)), np.ones((8, 2)), block=8)
