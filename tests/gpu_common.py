"""Shared helpers for the GPU parity tests (inputs and oracle references)."""
from __future__ import annotations

import numpy as np

import oracle
from paper_1807_10633_gb300 import systems as S


def make_case(name: str, W: int, seed: int = S.MASTER_SEED, **pk):
    sys_ = S.named_system(name)
    prm = S.make_params(sys_, seed=seed, **pk)
    occ = S.init_occupations(sys_, prm, W, seed=seed + 1)
    return sys_, prm, occ


def oracle_n(sys_, occ):
    return oracle.occ_lists_to_n(occ, sys_.M, sys_.n_alpha)


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.max(np.abs(a - b) / np.maximum(1.0, np.abs(b)))
