"""The synthetic inputs (paper_1807_10633_gb300/systems.py) against facts fixed outside this code:
the textbook STO-3G H2 energies, the symmetries of real two-electron integrals and the
orthonormality of the Loewdin orbitals.  CPU only."""
import numpy as np

from paper_1807_10633_gb300 import systems as S
from tests import brute


def test_h2_sto3g_energies_match_the_textbook():
    # Szabo & Ostlund, "Modern Quantum Chemistry", STO-3G H2 at R = 1.4 bohr (zeta = 1.24, the
    # exponents used here): SCF energy -1.1167 Eh, full CI -1.1373 Eh (four decimals printed).
    sys_ = S.hchain(2, spacing=1.4)
    assert abs(sys_.e_core - 1 / 1.4) < 1e-14
    c = np.array([1.0, 1.0]) / np.sqrt(2.0)          # sigma_g in the Loewdin basis
    e_scf = 2 * c @ sys_.h1 @ c + np.einsum("p,q,r,s,pqrs->", c, c, c, c, sys_.eri) + sys_.e_core
    _, H = brute.hamiltonian(sys_)
    Hd = H.toarray() if hasattr(H, "toarray") else np.asarray(H)
    e_fci = np.linalg.eigvalsh(Hd)[0]
    assert abs(e_scf - (-1.1167)) < 1.5e-4
    assert abs(e_fci - (-1.1373)) < 1.5e-4


def test_chain_integrals_are_symmetric_and_orbitals_orthonormal():
    sys_ = S.hchain(6)
    e = sys_.eri
    for perm in ("qprs", "pqsr", "rspq", "srqp"):
        np.testing.assert_allclose(e, np.einsum("pqrs->" + perm, e), atol=1e-12)
    np.testing.assert_allclose(sys_.h1, sys_.h1.T, atol=1e-12)
    assert sys_.n_alpha == sys_.n_beta == 3
    # (pp|qq) >= 0 and the Coulomb matrix is positive definite for real orbitals
    Jm = np.einsum("ppqq->pq", e)
    assert np.linalg.eigvalsh(Jm).min() > 0


def test_hubbard_ring_integrals():
    sys_ = S.hubbard(10, 1, t=1.0, U=4.0)
    h = sys_.h1
    for i in range(10):
        assert h[i, (i + 1) % 10] == -1.0 and h[i, (i - 1) % 10] == -1.0
    assert np.count_nonzero(h) == 20
    e = sys_.eri
    assert np.count_nonzero(e) == 10 and all(e[i, i, i, i] == 4.0 for i in range(10))
