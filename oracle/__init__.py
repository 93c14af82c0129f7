"""Oracle for the screened orbital-space VMC hot path -- TEST INFRASTRUCTURE ONLY.

A plain FP64 CPU implementation (``vmc_oracle.c``) of what the GPU path computes, written
from the paper (arXiv:1807.10633): the screened local energy of Sec. II.A, Eq. (eloc:hci);
the CTMC rates, residence time and choice of Sec. II.B, Eq. (rate); the gradient ratios of
Sec. III.B; AMSGrad, Eqs. (m1)-(m2) of Sec. II.C.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may use it.  It shares no code with the CUDA library
and never calls it.

Pins (tests that tie it to something other than itself) live in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "vmc_oracle.c"
_BUILD = _HERE / "_build"
_LIB = _BUILD / "liboracle.so"


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (plain C, OpenMP over walkers, no FP contraction)."""
    _BUILD.mkdir(exist_ok=True)
    if force or not _LIB.exists() or _LIB.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _BUILD / f"liboracle.{os.getpid()}.so"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                               "-ffp-contract=off", "-o", str(tmp), str(_SRC), "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _System(ct.Structure):
    _fields_ = [("M", ct.c_int), ("n_alpha", ct.c_int), ("n_beta", ct.c_int),
                ("h1", ct.c_void_p), ("eri", ct.c_void_p), ("e_core", ct.c_double),
                ("J", ct.c_void_p), ("Ca", ct.c_void_p), ("Cb", ct.c_void_p),
                ("n_corr", ct.c_int), ("corr_off", ct.c_void_p), ("corr_sites", ct.c_void_p),
                ("val_off", ct.c_void_p), ("corr_val", ct.c_void_p)]


MOVE_DTYPE = np.dtype([("kind", np.int32), ("i", np.int32), ("j", np.int32), ("a", np.int32),
                       ("b", np.int32), ("pad", np.int32), ("h", np.float64),
                       ("ratio", np.float64), ("key", np.float64)])

_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ct.CDLL(str(build()))
        P, D, L64, U64 = ct.c_void_p, ct.c_double, ct.c_long, ct.c_uint64
        L.orc_local_energy.argtypes = [P, P, D, ct.c_int, P, P, P, L64]
        L.orc_local_energy.restype = L64
        L.orc_local_energy_batch.argtypes = [P, L64, P, D, P, P, P, ct.c_int]
        L.orc_local_energy_batch.restype = L64
        L.orc_psi.argtypes = [P, P]
        L.orc_psi.restype = D
        L.orc_ctmc_choose.argtypes = [P, L64, U64, U64, U64, P, P]
        L.orc_ctmc_choose.restype = ct.c_int
        L.orc_ctmc_choose_u.argtypes = [P, L64, U64, P, P]
        L.orc_ctmc_choose_u.restype = ct.c_int
        L.orc_grad_logpsi.argtypes = [P, P, D, P, P, P]
        L.orc_grad_logpsi.restype = ct.c_int
        L.orc_grad_cps.argtypes = [P, P, D, P]
        L.orc_grad_cps.restype = None
        L.orc_amsgrad.argtypes = [P, P, P, P, L64, D, D, D]
        L.orc_amsgrad.restype = None
        L.orc_philox4x64.argtypes = [P, P, P]
        L.orc_philox4x64.restype = None
        L.orc_sweep.argtypes = [P, L64, P, D, U64, P, P, P, P, L64, ct.c_int]
        L.orc_sweep.restype = L64
        L.orc_near_ties.argtypes = [P, D]
        L.orc_near_ties.restype = L64
        _lib = L
    return _lib


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


def occ_lists_to_n(occ: np.ndarray, M: int, n_alpha: int) -> np.ndarray:
    """(W, n_e) occupied spatial orbitals (alpha block, then beta) -> (W, 2M) uint8 numbers."""
    occ = np.atleast_2d(occ)
    W = occ.shape[0]
    n = np.zeros((W, 2 * M), dtype=np.uint8)
    for w in range(W):
        n[w, occ[w, :n_alpha].astype(np.int64)] = 1
        n[w, M + occ[w, n_alpha:].astype(np.int64)] = 1
    return n


class Oracle:
    """FP64 oracle bound to one Hamiltonian and one set of wavefunction parameters; ``cps`` (a
    ``systems.CPS``) adds the correlator product of Sec. III.A to the pair Jastrow."""

    def __init__(self, system, params, cps=None):
        self.M = system.M
        self.n_alpha, self.n_beta = system.n_alpha, system.n_beta
        self._keep = dict(
            h1=np.ascontiguousarray(system.h1, dtype=np.float64),
            eri=np.ascontiguousarray(system.eri, dtype=np.float64),
            J=np.ascontiguousarray(params.J, dtype=np.float64),
            Ca=np.ascontiguousarray(params.C_alpha, dtype=np.float64),
            Cb=np.ascontiguousarray(params.C_beta, dtype=np.float64))
        k = self._keep
        n_corr = 0
        cp = [None] * 4
        if cps is not None and len(cps.sites):
            n_corr = len(cps.sites)
            k["corr_off"] = np.concatenate([[0], np.cumsum([len(x) for x in cps.sites])]).astype(np.int32)
            k["corr_sites"] = np.ascontiguousarray(np.concatenate(cps.sites), dtype=np.int32)
            k["val_off"] = np.concatenate([[0], np.cumsum([len(v) for v in cps.values])]).astype(np.int64)
            k["corr_val"] = np.ascontiguousarray(np.concatenate(cps.values), dtype=np.float64)
            for x, v in zip(cps.sites, cps.values):
                assert len(v) == 4 ** len(x) and np.all((0 <= np.asarray(x)) & (np.asarray(x) < self.M))
            cp = [_p(k["corr_off"]), _p(k["corr_sites"]), _p(k["val_off"]), _p(k["corr_val"])]
        self.n_corr_values = int(k["corr_val"].size) if n_corr else 0
        self._s = _System(self.M, self.n_alpha, self.n_beta, _p(k["h1"]), _p(k["eri"]),
                          float(system.e_core), _p(k["J"]), _p(k["Ca"]), _p(k["Cb"]), n_corr, *cp)
        self.move_cap = 1 << 16

    @property
    def sref(self):
        return ct.byref(self._s)

    def local_energy(self, n: np.ndarray, eps: float, direct: bool = False,
                     with_moves: bool = True):
        n = np.ascontiguousarray(n, dtype=np.uint8)
        el, ed = ct.c_double(), ct.c_double()
        cap = self.move_cap
        while True:
            mv = np.zeros(cap, dtype=MOVE_DTYPE) if with_moves else None
            nm = lib().orc_local_energy(self.sref, _p(n), eps, int(direct), ct.byref(el),
                                        ct.byref(ed), _p(mv) if with_moves else None, cap)
            if nm == -2:
                cap *= 4
                continue
            if nm < 0:
                raise ArithmeticError("singular determinant")
            break
        return el.value, ed.value, (mv[:nm] if with_moves else nm)

    def local_energy_batch(self, n: np.ndarray, eps: float, n_threads: int = 0):
        n = np.ascontiguousarray(n, dtype=np.uint8)
        W = n.shape[0]
        el = np.zeros(W)
        ed = np.zeros(W)
        nm = np.zeros(W, dtype=np.int64)
        nt = n_threads or os.cpu_count() or 1
        err = lib().orc_local_energy_batch(self.sref, W, _p(n), eps, _p(el), _p(ed), _p(nm), nt)
        if err:
            raise ArithmeticError(f"{err} walkers failed")
        return el, ed, nm

    def near_ties(self, eps: float) -> int:
        """Screening quantities (S_ia of same-spin singles, |<ab||ij>| of spin-conserving doubles, over
        all spin orbitals) within 1e-12 max(1, eps) of the threshold eps."""
        return int(lib().orc_near_ties(self.sref, float(eps)))

    def psi(self, n: np.ndarray) -> float:
        n = np.ascontiguousarray(n, dtype=np.uint8)
        return lib().orc_psi(self.sref, _p(n))

    def grad_logpsi(self, n: np.ndarray, weight: float, dJ, dCa, dCb):
        n = np.ascontiguousarray(n, dtype=np.uint8)
        rc = lib().orc_grad_logpsi(self.sref, _p(n), weight, _p(dJ), _p(dCa), _p(dCb))
        if rc:
            raise ArithmeticError("singular determinant")

    def grad_cps(self, n: np.ndarray, weight: float, dc: np.ndarray):
        """dc (all correlator coefficients, concatenated) += weight * d ln psi(n) / d c."""
        n = np.ascontiguousarray(n, dtype=np.uint8)
        assert dc.dtype == np.float64 and dc.flags.c_contiguous and dc.size == self.n_corr_values
        lib().orc_grad_cps(self.sref, _p(n), weight, _p(dc))

    def sweep(self, n: np.ndarray, eps: float, seed: int, steps: np.ndarray, n_threads: int = 0):
        """One CTMC step for every walker; n (W, 2M) and steps (W,) are updated in place."""
        assert n.dtype == np.uint8 and n.flags.c_contiguous
        assert steps.dtype == np.uint64 and steps.flags.c_contiguous
        W = n.shape[0]
        el = np.zeros(W)
        tr = np.zeros(W)
        mv = np.zeros((W, 5), dtype=np.int32)
        nt = n_threads or os.cpu_count() or 1
        err = lib().orc_sweep(self.sref, W, _p(n), eps, seed, _p(steps), _p(el), _p(tr), _p(mv),
                              self.move_cap, nt)
        return el, tr, mv, int(err)


def ctmc_choose(moves: np.ndarray, seed: int, walker: int, step: int):
    moves = np.ascontiguousarray(moves, dtype=MOVE_DTYPE)
    k = ct.c_long()
    t = ct.c_double()
    rc = lib().orc_ctmc_choose(_p(moves), moves.size, seed, walker, step, ct.byref(k), ct.byref(t))
    return rc, k.value, t.value


def ctmc_choose_u(moves: np.ndarray, U: int):
    """The choice rule for a given 64-bit uniform draw U (what ctmc_choose draws from Philox)."""
    moves = np.ascontiguousarray(moves, dtype=MOVE_DTYPE)
    k = ct.c_long()
    t = ct.c_double()
    rc = lib().orc_ctmc_choose_u(_p(moves), moves.size, U, ct.byref(k), ct.byref(t))
    return rc, k.value, t.value


def amsgrad(p, g, m, v, alpha, beta1, beta2):
    for a in (p, g, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lib().orc_amsgrad(_p(p), _p(g), _p(m), _p(v), p.size, alpha, beta1, beta2)


def philox4x64(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().orc_philox4x64(_p(c), _p(k), _p(out))
    return out
