"""Planted mistakes in the oracle: each is a one-line change to ``oracle/vmc_oracle.c``, compiled
from a patched copy in a temporary directory (the oracle itself is never edited), and at least
one pin of ``tests/test_oracle_pins.py`` must fail against it.  This checks that the pins would
catch a plausible slip anywhere in the oracle's arithmetic.  CPU only."""
import subprocess
from pathlib import Path

import pytest

import oracle
from paper_1807_10633_gb300 import systems as S
from tests import test_oracle_cps as C
from tests import test_oracle_pins as P

SRC = Path(oracle.__file__).with_name("vmc_oracle.c")


def _brute_h4():
    P.test_eloc_eps0_matches_brute_hchain(P._h4)


def _cps_brute_h4():
    C.test_cps_eloc_eps0_matches_brute_all_dets(lambda: S.hchain(4))


# (mistake, exact source line fragment, replacement, the pin that must fail)
MUTANTS = [
    ("exchange sign in <pq||rs>",
     "return phys(s, p, q, r, t) - phys(s, p, q, t, r);",
     "return phys(s, p, q, r, t) + phys(s, p, q, t, r);", _brute_h4),
    ("canonical phase dropped from doubles",
     "double hel = ph * v;", "double hel = v;", _brute_h4),
    ("two-electron part of the single's matrix element dropped",
     "if (n[j]) hel += phys_anti(s, a, j, i, j);", "if (0) hel += phys_anti(s, a, j, i, j);", _brute_h4),
    ("exchange dropped from the diagonal energy",
     "ed += 0.5 * phys_anti(s, i, j, i, j);", "ed += 0.5 * phys(s, i, j, i, j);", _brute_h4),
    ("one-body Jastrow term dropped",
     "acc += s->J[(size_t)p * N2 + p];", "acc += 0.0;", _brute_h4),
    ("two-electron bound dropped from S_ia",
     "acc += fabs(phys(s, i, j, a, j) - phys(s, i, j, j, a));", "acc += 0.0;",
     P.test_singles_screen_uses_two_electron_bound),
    ("transposed inverse index in d ln det / d theta",
     "t.Ainv[sg][(size_t)x * ns + r]", "t.Ainv[sg][(size_t)r * ns + x]",
     P.test_grad_logpsi_matches_finite_differences),
    ("nine Philox rounds instead of ten",
     "for (int r = 0; r < 10; ++r) {", "for (int r = 0; r < 9; ++r) {",
     lambda: P.test_philox_matches_numpy((1807, 123456), (99, 1, 2, 3))),
    ("CTMC choice uniform over moves instead of by rate",
     "pre += rate_fixed(fabs(moves[k].ratio));", "pre += Q / (u128)nm;", P.test_ctmc_choice_distribution),
    ("first non-zero pivot instead of the largest in the LU",
     "if (v > best) { best = v; p = r; }", "if (best == 0.0 && v > best) { best = v; p = r; }",
     P.test_table_ratios_with_a_tiny_leading_pivot),
    ("choice rule takes the first prefix at or above T instead of above it",
     "if (pre > T) { *chosen = k; return 0; }", "if (pre >= T) { *chosen = k; return 0; }",
     P.test_ctmc_choice_rule_at_exact_boundaries),
    ("integer part of Q dropped from T = floor(U Q / 2^64)",
     "u128 T = (u128)U * qh + (u128)(((u128)U * ql) >> 64);", "u128 T = (u128)(((u128)U * ql) >> 64);",
     P.test_ctmc_choice_rule_at_exact_boundaries),
    ("residence time not inverted",
     "*t_res = 1.0 / ((double)qh + (double)ql * 0x1p-64);", "*t_res = (double)qh + (double)ql * 0x1p-64;",
     P.test_ctmc_choice_distribution),
    ("row-exchange sign dropped from the LU determinant",
     "            sgn = -sgn;\n", "\n", P.test_direct_ratios_equal_table_ratios),
    ("sorting parity dropped from the in-place ratio",
     "return (inv & 1) ? -minor : minor;", "return minor;", _brute_h4),
    ("transposed inverse in G = C C_occ^-1",
     "acc += C[(size_t)k * ns + x] * t->Ainv[sg][(size_t)x * ns + cc];",
     "acc += C[(size_t)k * ns + x] * t->Ainv[sg][(size_t)cc * ns + x];", _brute_h4),
    ("forward substitution skips the last column of L",
     "for (int c = 0; c < r; ++c) b[r] -= work[(size_t)r * n + c] * b[c];",
     "for (int c = 0; c < r - 1; ++c) b[r] -= work[(size_t)r * n + c] * b[c];", _brute_h4),
    ("E_core dropped from the diagonal energy",
     "double ed = s->e_core;", "double ed = 0.0;", _brute_h4),
    ("one-body Jastrow term dropped from the gradient",
     "dJ[(size_t)p * N2 + p] += weight;", "dJ[(size_t)p * N2 + p] += 0.0;",
     P.test_energy_gradient_matches_exact_derivative),
    ("Philox Weyl constant off by one",
     "W1 = 0xBB67AE8584CAA73BULL", "W1 = 0xBB67AE8584CAA73AULL",
     lambda: P.test_philox_matches_numpy((1807, 123456), (99, 1, 2, 3))),
    ("fixed-point rate with 52 instead of 53 bits",
     "(uint64_t)ldexp(f, 53);", "(uint64_t)ldexp(f, 52);", P.test_ctmc_choice_distribution),
    ("alpha and beta swapped in a correlator's site state",
     "idx += w * (n[site] + 2 * n[s->M + site]);", "idx += w * (2 * n[site] + n[s->M + site]);",
     C.test_pair_jastrow_written_as_correlators_gives_the_same_energies),
    ("correlator digits in base 2 instead of 4",
     "++e, w *= 4)", "++e, w *= 2)", _cps_brute_h4),
    ("correlator ratio left out of the doubles",
     "spin_ratio(&t, 1, 1, &fb, &tb, M) * jr;\n                        }\n"
     "                        if (s->n_corr) ratio *= cps_value(s, m) / cps_n;",
     "spin_ratio(&t, 1, 1, &fb, &tb, M) * jr;\n                        }", _cps_brute_h4),
    ("d ln psi / d c without the 1/c",
     "dc[k] += weight / s->corr_val[k];", "dc[k] += weight;", C.test_cps_gradient_matches_finite_differences),
    ("AMSGrad without the running maximum",
     "v[k] = v[k] > cand ? v[k] : cand;", "v[k] = cand;", P.test_amsgrad_hand_recurrence),
    ("AMSGrad with the usual (not the paper's) beta1 convention",
     "m[k] = (1.0 - beta1) * m[k] + beta1 * g[k];", "m[k] = beta1 * m[k] + (1.0 - beta1) * g[k];",
     P.test_amsgrad_hand_recurrence),
]


@pytest.mark.parametrize("name,old,new,pin", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(tmp_path, monkeypatch, name, old, new, pin):
    src = SRC.read_text()
    assert src.count(old) == 1, f"the mutation site of '{name}' is not unique or has moved"
    mutant = tmp_path / "mutant.c"
    mutant.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                           "-o", str(so), str(mutant), "-lm"])
    monkeypatch.setattr(oracle, "build", lambda force=False: so)
    monkeypatch.setattr(oracle, "_lib", None)
    with pytest.raises(AssertionError):
        pin()


def test_unmutated_oracle_passes_the_same_pins():
    for _, _, _, pin in MUTANTS:
        pin()
