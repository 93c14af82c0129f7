"""Checkpoint and resume of the optimisation loop (Sec. II.C).

A checkpoint holds what the next iteration needs and the library cannot recompute bit for bit:
- the flat parameters p, the AMSGrad moments m and v (Eqs. m1-m2) and the index of the next
  iteration (which fixes the step-size schedule and the CTMC seed word);
- per walker: the occupied orbitals in their current column order (moves replace an orbital in
  place, so this order fixes the column order of C_occ and with it the rounding of every table
  built from it), the Philox step counter, the diagonal energy E_diag and the Fock sums F (both
  updated per move);
- the correlator sites when the wavefunction has a correlator product;
- what the tables belong to: W, M, n_alpha, n_beta, the precision form, the screening threshold,
  and a digest of the one-electron integrals and the core energy.

`load` builds the engine from the saved occupations and parameters, which forms G, C_occ^-1, the
Jastrow sums and the correlator indices with the same kernels and inputs as the table refresh that
ends an iteration, then restores E_diag, F and the counters.  A checkpoint written between
iterations therefore continues bit-identically to an uninterrupted run; one written after some
sweeps of an iteration continues from tables recomputed from the occupations, as a refresh would
leave them.

The file is a plain numpy .npz archive; the integrals themselves are not stored (the caller passes
the same system again, and the digest check rejects a different one).
"""
from __future__ import annotations

import hashlib
from pathlib import Path

import numpy as np
import torch

from . import systems as S
from . import vmc
from .optimize import OptState

FORMAT = 1


def system_digest(system) -> str:
    """sha-256 of the one-electron integrals, the core energy and the electron counts."""
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(system.h1, dtype=np.float64).tobytes())
    h.update(np.array([system.e_core], dtype=np.float64).tobytes())
    h.update(np.array([system.M, system.n_alpha, system.n_beta], dtype=np.int64).tobytes())
    return h.hexdigest()


def save(path, eng: vmc.Engine, state: OptState, system) -> Path:
    """Write the checkpoint of `eng` (parameters and walkers, built on `system`) and `state`."""
    if system.M != eng.M or system.n_alpha != eng.na or system.n_beta != eng.nb:
        raise ValueError("the system does not match the engine")
    if eng.p.is_cuda:
        torch.cuda.synchronize(eng.p.device)
    w = eng.walkers
    arrays = {
        "format": np.array(FORMAT),
        "shape": np.array([eng.W, eng.M, eng.na, eng.nb, w.precision], dtype=np.int64),
        "eps": np.array(eng.eps, dtype=np.float64),
        "digest": np.array(system_digest(system)),
        "p": eng.p.detach().cpu().numpy(),
        "m": state.m.detach().cpu().numpy(),
        "v": state.v.detach().cpu().numpy(),
        "next_iter": np.array(state.next_iter, dtype=np.int64),
        "occ_list": w.occ_list.cpu().numpy().reshape(eng.W, eng.na + eng.nb),
        "rng_counter": w.rng_counter.cpu().numpy(),
        "e_diag": w.e_diag.cpu().numpy(),
        "F": w.F.cpu().numpy(),
    }
    if eng.cps_sites is not None:
        arrays["cps_site_off"] = np.cumsum([0] + [len(s) for s in eng.cps_sites]).astype(np.int64)
        arrays["cps_sites"] = np.array([x for s in eng.cps_sites for x in s], dtype=np.int64)
    path = Path(path)
    with open(path, "wb") as f:          # a file object keeps the name as given (no ".npz" added)
        np.savez(f, **arrays)
    return path


def read(path, system) -> dict:
    """The checkpoint's arrays, after checking its format and that it was written for `system`."""
    with np.load(Path(path), allow_pickle=False) as z:
        ck = {k: z[k] for k in z.files}
    if int(ck["format"]) != FORMAT:
        raise ValueError(f"checkpoint format {int(ck['format'])}, expected {FORMAT}")
    W, M, na, nb, precision = (int(x) for x in ck["shape"])
    if (M, na, nb) != (system.M, system.n_alpha, system.n_beta) or str(ck["digest"]) != system_digest(system):
        raise ValueError("the checkpoint was written for a different system")
    if precision not in (vmc.VMC_FP64, vmc.VMC_MIXED):
        raise ValueError("bad precision form in the checkpoint")
    n_j, n_c = (2 * M) ** 2, M * (na + nb)
    n_cps = int(ck["p"].size) - n_j - n_c
    if n_cps < 0 or ck["m"].shape != ck["p"].shape or ck["v"].shape != ck["p"].shape:
        raise ValueError("inconsistent parameter arrays in the checkpoint")
    if (n_cps > 0) != ("cps_sites" in ck):
        raise ValueError("correlator coefficients without correlator sites (or the reverse)")
    if ck["occ_list"].shape != (W, na + nb) or ck["rng_counter"].size != W or ck["e_diag"].size != W:
        raise ValueError("inconsistent walker arrays in the checkpoint")
    return ck


def wavefunction(ck: dict) -> tuple[S.Params, S.CPS | None]:
    """The parameters of a checkpoint split back into J, C_alpha, C_beta and the correlators."""
    W, M, na, nb, _ = (int(x) for x in ck["shape"])
    p = ck["p"]
    n_j, n_a, n_b = (2 * M) ** 2, M * na, M * nb
    prm = S.Params(p[:n_j].reshape(2 * M, 2 * M).copy(), p[n_j:n_j + n_a].reshape(M, na).copy(),
                   p[n_j + n_a:n_j + n_a + n_b].reshape(M, nb).copy())
    if "cps_sites" not in ck:
        return prm, None
    off, flat = ck["cps_site_off"], ck["cps_sites"]
    sites = [[int(x) for x in flat[off[l]:off[l + 1]]] for l in range(off.size - 1)]
    vals, k = [], n_j + n_a + n_b
    for st in sites:
        vals.append(p[k:k + 4 ** len(st)].copy())
        k += 4 ** len(st)
    if k != p.size:
        raise ValueError("correlator coefficients do not match the correlator sites")
    return prm, S.CPS(sites, vals)


def load(path, system, device: int = 0, stream=None) -> tuple[vmc.Engine, OptState]:
    """Rebuild the engine and the optimiser state of a checkpoint written by `save` for `system`."""
    ck = read(path, system)
    precision = int(ck["shape"][4])
    p = ck["p"]
    prm, cps = wavefunction(ck)
    eng = vmc.Engine(system, prm, ck["occ_list"], eps=float(ck["eps"]), precision=precision, device=device,
                     stream=stream, cps=cps)
    dev = eng.p.device
    torch.cuda.synchronize(dev)          # the table build (on the engine's stream) is done
    if not np.array_equal(eng.p.cpu().numpy(), p):
        raise ValueError("the rebuilt parameters differ from the checkpoint's")
    w = eng.walkers
    if w.F.numel() != ck["F"].size:
        raise ValueError("Fock-sum array of the checkpoint does not match the screened lists")
    w.e_diag.copy_(torch.from_numpy(ck["e_diag"]))
    w.F.copy_(torch.from_numpy(ck["F"]))
    w.rng_counter.copy_(torch.from_numpy(ck["rng_counter"]))
    state = OptState(torch.from_numpy(ck["m"]).to(dev), torch.from_numpy(ck["v"]).to(dev), int(ck["next_iter"]))
    torch.cuda.synchronize(dev)
    return eng, state
