"""Host pass of the screened-list builder through the C ABI (CPU only, no device needed):
8-fold packed and dense integrals give bit-identical lists, and the builder's near-tie count of the
threshold (Sec. II.A keeps |x| > eps) equals the oracle's, which is pinned to a closed form."""
import numpy as np
import pytest

import oracle
from paper_1807_10633_gb300 import systems as S
from paper_1807_10633_gb300 import vmc


@pytest.mark.parametrize("name", ["hubbard4x4", "H20", "H80"])
@pytest.mark.parametrize("eps", [1e-6, 1e-4])
def test_packed_and_dense_integrals_give_identical_lists(name, eps):
    sys_ = S.named_system(name)
    packed = S.pack_eri(sys_.eri)
    assert packed.size == (sys_.M * (sys_.M + 1) // 2) * (sys_.M * (sys_.M + 1) // 2 + 1) // 2
    dense = vmc.vmc_screened_lists_summary(sys_.M, sys_.h1, sys_.eri, eps)
    pk = vmc.vmc_screened_lists_summary(sys_.M, sys_.h1, packed, eps)
    assert dense == pk
    assert dense["singles"] > 0


def test_pack_round_trip_is_exact_on_symmetric_integrals():
    sys_ = S.named_system("H20")
    np.testing.assert_array_equal(S.unpack_eri(S.pack_eri(sys_.eri), sys_.M), sys_.eri)


def _ring_near_ties(M, eps):
    """Closed form for the periodic Hubbard ring (t = 1, U = 4, M > 2): every S_ia is t for the 2M
    neighbour pairs and 0 otherwise; every |<ab||ij>| with a, b outside {i, j} is 0 (the only
    non-zero two-electron integral is (pp|pp))."""
    singles_t, singles_0 = 2 * (2 * M), 2 * (M * (M - 1) - 2 * M)
    doubles_0 = 2 * (M * (M - 1) // 2) * ((M - 2) * (M - 3) // 2) + M * M * (M - 1) * (M - 1)
    return {0.0: singles_0 + doubles_0, 1.0: singles_t, 0.5: 0}[eps]


@pytest.mark.parametrize("eps", [0.0, 1.0, 0.5])
def test_oracle_near_ties_match_the_hubbard_closed_form(eps):
    sys_ = S.hubbard(10)
    orc = oracle.Oracle(sys_, S.make_params(sys_))
    assert orc.near_ties(eps) == _ring_near_ties(10, eps)


def _opposite_spin_key(sys_):
    """A magnitude that is exactly one opposite-spin double's screening key, |(ap|bq)|."""
    a, p, b, q = 2, 3, 5, 4
    return abs(float(sys_.eri[a, p, b, q]))


@pytest.mark.parametrize("name,eps", [("hubbard10", 0.0), ("hubbard10", 1.0), ("H6", 1e-6), ("H20", 1e-6),
                                      ("H20", "key")])
def test_builder_near_ties_equal_the_oracle(name, eps):
    sys_ = S.named_system(name)
    if eps == "key":
        eps = _opposite_spin_key(sys_)
    orc = oracle.Oracle(sys_, S.make_params(sys_))
    want = orc.near_ties(eps)
    got = vmc.vmc_screened_lists_summary(sys_.M, sys_.h1, sys_.eri, eps)["near_ties"]
    assert got == want
    if name == "H20" and eps > 1e-4:
        assert want >= 1           # the chosen key is itself a near tie
