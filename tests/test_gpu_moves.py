"""The screened move set, element by element, against the oracle's enumeration (needs a GB300).

For each sampled walker the library's vmc_screened_moves lists every connected determinant that
survives the screen of Sec. II.A (heat-bath lists cut at eps_run) with empty targets, in the
canonical order of the CTMC choice (Sec. II.B).  The oracle enumerates the same excitations from the
integral tensor itself, with canonical fermionic phases.  Checked: the move codes (kind, i, j, a, b)
and their order bit-exactly, in both precision forms; |psi(m)/psi(n)| (the CTMC rate) and
H_nm psi(m)/psi(n) element by element (FP64 form 1e-10); the walked list entries against counts
made from the integrals in numpy; and the near-tie count of the threshold on both sides.
"""
from concurrent.futures import ThreadPoolExecutor
import os

import numpy as np
import pytest

import oracle
from paper_1807_10633_gb300 import systems as S
from tests.gpu_common import oracle_n

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vmc():
    from paper_1807_10633_gb300 import vmc as v
    v.lib()
    return v


_SYSTEMS = {}


def _system(name):
    if name not in _SYSTEMS:
        _SYSTEMS[name] = S.named_system(name)
    return _SYSTEMS[name]


def _oracle_moves(orc, n, eps_run):
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:   # the oracle call releases the GIL
        return list(ex.map(lambda x: orc.local_energy(x, eps_run), list(n)))


def _walked_counts(sys_, occ, eps_run):
    """List entries a walk over occupied pairs reads, from the integrals (numpy): singles lists of
    occupied orbitals and double lists of occupied pairs, each entry counted whether or not its
    targets are empty."""
    M, na = sys_.M, sys_.n_alpha
    e = sys_.eri
    Jt = np.einsum("iakk->iak", e)
    Kt = np.einsum("ikka->iak", e)
    Sia = np.abs(sys_.h1) + np.abs(Jt - Kt).sum(-1) + np.abs(Jt).sum(-1)
    np.fill_diagonal(Sia, 0.0)
    s_len = (Sia > eps_run).sum(axis=1)
    ab = np.ones((M, M), dtype=bool)
    out = []
    for w in range(occ.shape[0]):
        oa, ob = occ[w, :na].astype(int), occ[w, na:].astype(int)
        ws = int(s_len[oa].sum() + s_len[ob].sum())
        wd = 0
        for spin_occ in (oa, ob):
            for x in range(len(spin_occ)):
                for y in range(x + 1, len(spin_occ)):
                    p, q = sorted((spin_occ[x], spin_occ[y]))
                    v = e[:, p, :, q] - e[:, q, :, p]          # v[a, b] = (ap|bq) - (aq|bp)
                    m = np.triu(ab, 1).copy()
                    m[[p, q], :] = False
                    m[:, [p, q]] = False
                    wd += int((np.abs(v[m]) > eps_run).sum())
        for p in oa:
            for q in ob:
                v = e[:, p, :, q].copy()
                v[p, :] = 0.0
                v[:, q] = 0.0
                wd += int((np.abs(v) > eps_run).sum())
        out.append((ws, wd))
    return np.array(out)


def _check_walker(vmc, ref, got, precision, e_loc_gpu, e_diag, n_elec):
    el_ref, _, mv = ref
    code, ratio, contrib = got
    want = np.stack([mv["kind"], mv["i"], mv["j"], mv["a"], mv["b"]], axis=1).astype(np.int64)
    have = vmc.decode_moves(code)
    assert have.shape == want.shape, (have.shape, want.shape)
    np.testing.assert_array_equal(have, want)
    r_ref = np.abs(mv["ratio"])
    c_ref = mv["h"] * mv["ratio"]
    rmax, cmax = max(1e-300, r_ref.max()), max(1e-300, np.abs(c_ref).max())
    if precision == vmc.VMC_FP64:
        assert np.all(np.abs(np.abs(ratio) - r_ref) <= 1e-10 * (r_ref + 1e-3 * rmax))
        assert np.all(np.abs(contrib - c_ref) <= 1e-10 * (np.abs(c_ref) + 1e-3 * cmax))
        assert abs(e_diag + contrib.sum() - el_ref) <= 1e-10 * max(1.0, abs(el_ref))
        assert abs(e_diag + contrib.sum() - e_loc_gpu) <= 1e-10 * max(1.0, abs(el_ref))
    else:
        assert np.all(np.abs(np.abs(ratio) - r_ref) <= 1e-3 * (r_ref + 1e-2 * rmax))
        assert abs(e_diag + contrib.sum() - el_ref) < 1e-4 * n_elec   # 0.1 mEh per electron


# (system, build eps, walkers, sampled walkers, eps_run values, packed integrals)
CASES = [("hubbard10", 0.0, 256, 256, (0.0, 0.5), False),
         ("H20", 1e-6, 512, 64, (1e-6, 3e-5), False),
         ("H80", 1e-6, 1024, 12, (1e-6, 1e-4), True),
         ("H160", 1e-6, 256, 4, (1e-6, 1e-5), True)]


@pytest.mark.parametrize("name,eps,W,n_check,eps_runs,packed", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_screened_moves_match_the_oracle(vmc, name, eps, W, n_check, eps_runs, packed, form):
    precision = vmc.VMC_FP64 if form == "fp64" else vmc.VMC_MIXED
    sys_ = _system(name)
    prm = S.make_params(sys_, seed=S.MASTER_SEED)
    occ = S.init_occupations(sys_, prm, W, seed=S.MASTER_SEED + 1)
    gpu_sys = S.System(sys_.name, sys_.M, sys_.n_alpha, sys_.n_beta, sys_.h1,
                       S.pack_eri(sys_.eri) if packed else sys_.eri, sys_.e_core)
    eng = vmc.Engine(gpu_sys, prm, occ, eps=eps, precision=precision)
    orc = oracle.Oracle(sys_, prm)
    idx = np.linspace(0, W - 1, n_check).astype(int)
    n = np.ascontiguousarray(oracle_n(sys_, occ[idx]))
    try:
        for eps_run in eps_runs:
            e_loc, _ = eng.local_energy(eps_run)
            eng.sync()
            e_loc = e_loc.cpu().numpy()
            e_diag = eng.walkers.e_diag.cpu().numpy()
            refs = _oracle_moves(orc, n, eps_run)
            for k, w in enumerate(idx):
                per, cnt, walked = eng.screened_moves(int(w), 1, eps_run)
                eng.sync()
                assert cnt[0] == len(refs[k][2])
                assert walked[0, 0] + walked[0, 1] >= cnt[0]
                _check_walker(vmc, refs[k], per[0], precision, e_loc[w], e_diag[w], sys_.n_elec)
            if name in ("hubbard10", "H20") and form == "fp64":
                per, cnt, walked = eng.screened_moves(int(idx[0]), 8, eps_run)
                np.testing.assert_array_equal(walked, _walked_counts(sys_, occ[idx[0]:idx[0] + 8], eps_run))
    finally:
        eng.close()


@pytest.mark.parametrize("name,eps", [("hubbard10", 0.0), ("hubbard10", 1.0), ("H20", 1e-6), ("H80", 1e-6)])
def test_near_ties_of_the_device_lists_equal_the_oracle(vmc, name, eps):
    sys_ = _system(name)
    prm = S.make_params(sys_, seed=S.MASTER_SEED)
    occ = S.init_occupations(sys_, prm, 4, seed=S.MASTER_SEED + 1)
    eng = vmc.Engine(sys_, prm, occ, eps=eps, precision=vmc.VMC_FP64)
    try:
        got = vmc.vmc_lists_near_ties(eng.lists, eps)
        assert got == oracle.Oracle(sys_, prm).near_ties(eps)
        if name.startswith("H"):       # above the build eps: counted from the stored entries
            assert vmc.vmc_lists_near_ties(eng.lists, 10 * eps) == oracle.Oracle(sys_, prm).near_ties(10 * eps)
    finally:
        eng.close()


def test_h160_lists_from_packed_and_dense_integrals_are_identical(vmc):
    sys_ = _system("H160")
    dense = vmc.vmc_screened_lists_summary(sys_.M, sys_.h1, sys_.eri, 1e-6)
    packed = vmc.vmc_screened_lists_summary(sys_.M, sys_.h1, S.pack_eri(sys_.eri), 1e-6)
    assert dense == packed
    assert (dense["singles"], dense["same"], dense["opposite"]) == (3388, 30404, 129640)
