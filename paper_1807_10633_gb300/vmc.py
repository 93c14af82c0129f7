"""Python binding of the C ABI in include/vmc.h (argument marshalling only).

Every function here forwards to the CUDA library ``_build/libvmc.so``; nothing is computed in
Python.  PyTorch provides device memory (tensors) and streams.  If the library has not been
built the import of this module succeeds but every call raises ``RuntimeError``: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as ct
from dataclasses import dataclass

import numpy as np
import torch

from .build import LIB

VMC_FP64, VMC_MIXED = 0, 1
VMC_OPT_G_TENSOR_CORES, VMC_OPT_ELOC_THREADS, VMC_OPT_REFRESH_SMEM, VMC_OPT_MIXED_REFRESH_GJ32 = 1, 2, 3, 4
VMC_OPT_GRAD_J_TENSOR_CORES = 5
_STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_OOM", 4: "ERR_SINGULAR", 5: "ERR_TIMEOUT",
           6: "ERR_OVERFLOW", 7: "ERR_NOMOVE"}


class VmcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"vmc {_STATUS.get(status, status)}: {msg}")
        self.status = status


class vmc_walkers(ct.Structure):
    _fields_ = [("W", ct.c_int), ("M", ct.c_int), ("n_alpha", ct.c_int), ("n_beta", ct.c_int),
                ("precision", ct.c_int),
                ("occ_bits", ct.c_void_p), ("occ_list", ct.c_void_p), ("virt_list", ct.c_void_p),
                ("pos", ct.c_void_p), ("G", ct.c_void_p), ("AinvT", ct.c_void_p), ("S", ct.c_void_p), ("F", ct.c_void_p),
                ("e_diag", ct.c_void_p), ("rng_counter", ct.c_void_p), ("cps_state", ct.c_void_p)]


class vmc_params(ct.Structure):
    _fields_ = [("J", ct.c_void_p), ("C_alpha", ct.c_void_p), ("C_beta", ct.c_void_p),
                ("cps", ct.c_void_p), ("cps_values", ct.c_void_p)]


class vmc_batch_item(ct.Structure):
    _fields_ = [("lists", ct.c_void_p), ("params", ct.POINTER(vmc_params)), ("walkers", ct.POINTER(vmc_walkers)),
                ("eps_run", ct.c_double), ("d_e_loc", ct.c_void_p), ("d_t_res", ct.c_void_p),
                ("d_move_code", ct.c_void_p)]


_lib = None


def lib() -> ct.CDLL:
    """The loaded CUDA library; raises if it is missing (no fallback)."""
    global _lib
    if _lib is None:
        if not LIB.exists():
            raise RuntimeError(f"CUDA library {LIB} is not built; run __graft_entry__.build()")
        L = ct.CDLL(str(LIB))
        P, I, D, U64, I64 = ct.c_void_p, ct.c_int, ct.c_double, ct.c_uint64, ct.c_int64
        sig = {
            "vmc_create": ([ct.POINTER(P), I, P], I),
            "vmc_destroy": ([P], I),
            "vmc_set_stream": ([P, P], I),
            "vmc_last_error": ([P], ct.c_char_p),
            "vmc_sync": ([P], I),
            "vmc_build_screened_lists": ([P, I, P, P, I, D, D, ct.POINTER(P)], I),
            "vmc_screened_lists_summary": ([I, P, P, I, D, ct.POINTER(I64)], I),
            "vmc_lists_near_ties": ([P, D, ct.POINTER(I64)], I),
            "vmc_lists_layout": ([P, ct.POINTER(I), ct.POINTER(I)], I),
            "vmc_screened_moves": ([P, P, ct.POINTER(vmc_params), ct.POINTER(vmc_walkers), D, I, I, I64,
                                    P, P, P, P, P], I),
            "vmc_lists_destroy": ([P], I),
            "vmc_lists_info": ([P, ct.POINTER(I64), ct.POINTER(I64), ct.POINTER(I64)], I),
            "vmc_walkers_sizes": ([I, I, I, I, P, ct.POINTER(I64)], I),
            "vmc_walkers_init": ([P, P, ct.POINTER(vmc_params), ct.POINTER(vmc_walkers)], I),
            "vmc_walkers_refresh": ([P, P, ct.POINTER(vmc_params), ct.POINTER(vmc_walkers)], I),
            "vmc_log_psi": ([P, ct.POINTER(vmc_walkers), ct.POINTER(vmc_params), P], I),
            "vmc_local_energy": ([P, P, ct.POINTER(vmc_params), ct.POINTER(vmc_walkers), D, P, P], I),
            "vmc_ctmc_step": ([P, P, ct.POINTER(vmc_params), ct.POINTER(vmc_walkers), U64, P], I),
            "vmc_grad_logpsi": ([P, ct.POINTER(vmc_walkers), P, P, P, P], I),
            "vmc_amsgrad_update": ([P, P, P, P, P, ct.c_size_t, D, D, D], I),
            "vmc_walker_reduce": ([P, I, P, P, P], I),
            "vmc_energy_gradient": ([P, ct.c_size_t, P, P, P, P], I),
            "vmc_accumulate_gradient": ([P, ct.POINTER(vmc_walkers), P, P, P, P, P, P, P, P, P], I),
            "vmc_launch_count": ([P], U64),
            "vmc_probe_l2_read": ([P, P, ct.c_size_t, I], I),
            "vmc_cps_create": ([P, I, I, P, P, ct.POINTER(P)], I),
            "vmc_cps_destroy": ([P], I),
            "vmc_cps_info": ([P, ct.POINTER(I), ct.POINTER(I64)], I),
            "vmc_grad_logpsi_cps": ([P, ct.POINTER(vmc_walkers), ct.POINTER(vmc_params), P, P], I),
            "vmc_accumulate_gradient_cps": ([P, ct.POINTER(vmc_walkers), ct.POINTER(vmc_params), P, P, P, P], I),
            "vmc_set_option": ([P, I, I], I),
            "vmc_grad_logpsi_noalloc": ([ct.POINTER(vmc_walkers), P, P, P, P, P], I),
            "vmc_local_energy_batch": ([P, I, ct.POINTER(vmc_batch_item)], I),
            "vmc_ctmc_step_batch": ([P, I, ct.POINTER(vmc_batch_item), U64], I),
            "vmc_autotune_local_energy": ([P, I, ct.POINTER(vmc_batch_item), ct.POINTER(I)], I),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        if not t.is_contiguous():
            raise ValueError("tensors passed to the library must be contiguous")
        return t.data_ptr()
    if isinstance(t, np.ndarray):
        if not t.flags.c_contiguous:
            raise ValueError("arrays passed to the library must be C-contiguous")
        return t.ctypes.data
    return int(t)


_F64 = (torch.float64,)
_CODES = (torch.int64,) + ((torch.uint64,) if hasattr(torch, "uint64") else ())


def _need(t, name: str, n: int, dtypes=_F64):
    """Check a device-tensor argument before its pointer crosses the ABI, where a wrong dtype, size
    or device would let a kernel read or write past the buffer.  None (an absent optional output)
    and raw integer pointers pass unchecked: the caller vouches for those."""
    if t is None or isinstance(t, int):
        return
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name}: expected a CUDA tensor, got {type(t).__name__}")
    if t.dtype not in dtypes:
        raise ValueError(f"{name}: dtype {t.dtype}, expected {' or '.join(map(str, dtypes))}")
    if t.numel() < n:
        raise ValueError(f"{name}: {t.numel()} elements, at least {n} needed")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    if not t.is_cuda:
        raise ValueError(f"{name}: must be a CUDA tensor")


def _need_grad(walkers, dJ, dCa, dCb, prefix=""):
    N2 = 2 * walkers.M
    _need(dJ, prefix + "dJ", N2 * N2)
    _need(dCa, prefix + "dC_alpha", walkers.M * walkers.n_alpha)
    _need(dCb, prefix + "dC_beta", walkers.M * walkers.n_beta)


def _check(ctx, st: int):
    if st != 0:
        msg = lib().vmc_last_error(ctx).decode() if ctx else ""
        raise VmcError(st, msg)


# ------------------------------------------------------------------ raw C-ABI wrappers
def vmc_create(device: int = 0, stream=None):
    ctx = ct.c_void_p()
    s = stream.cuda_stream if isinstance(stream, torch.cuda.Stream) else (stream or 0)
    _check(None, lib().vmc_create(ct.byref(ctx), device, s))
    return ctx


def vmc_destroy(ctx):
    lib().vmc_destroy(ctx)


def vmc_set_stream(ctx, stream):
    s = stream.cuda_stream if isinstance(stream, torch.cuda.Stream) else (stream or 0)
    _check(ctx, lib().vmc_set_stream(ctx, s))


def vmc_last_error(ctx) -> str:
    return lib().vmc_last_error(ctx).decode()


def vmc_sync(ctx):
    _check(ctx, lib().vmc_sync(ctx))


def eri_form(M: int, eri: np.ndarray) -> int:
    """0 for dense (pq|rs) [M^4] storage, 1 for the 8-fold packed form (see include/vmc.h)."""
    npair = M * (M + 1) // 2
    if eri.size == M ** 4:
        return 0
    if eri.size == npair * (npair + 1) // 2:
        return 1
    raise ValueError(f"eri: {eri.size} elements is neither M^4 nor the 8-fold packed size for M = {M}")


def _integrals(M, h1, eri):
    h1 = np.ascontiguousarray(h1, dtype=np.float64)
    eri = np.ascontiguousarray(eri, dtype=np.float64)
    if h1.size != M * M:
        raise ValueError(f"h1: {h1.size} elements, expected {M * M}")
    return h1, eri, eri_form(M, eri)


def vmc_build_screened_lists(ctx, M: int, h1: np.ndarray, eri: np.ndarray, e_core: float, eps: float):
    """eri dense [M^4] or 8-fold packed (detected from its size)."""
    h1, eri, packed = _integrals(M, h1, eri)
    out = ct.c_void_p()
    _check(ctx, lib().vmc_build_screened_lists(ctx, M, _ptr(h1), _ptr(eri), packed, float(e_core), float(eps),
                                               ct.byref(out)))
    return out


def vmc_screened_lists_summary(M: int, h1: np.ndarray, eri: np.ndarray, eps: float) -> dict:
    """Host pass of the list builder (no device): sizes, near ties and a digest of the lists."""
    h1, eri, packed = _integrals(M, h1, eri)
    out = (ct.c_int64 * 5)()
    st = lib().vmc_screened_lists_summary(M, _ptr(h1), _ptr(eri), packed, float(eps), out)
    if st != 0:
        raise VmcError(st, "vmc_screened_lists_summary")
    return dict(singles=out[0], same=out[1], opposite=out[2], near_ties=out[3], digest=out[4] & (2 ** 64 - 1))


def vmc_lists_layout(lists) -> dict:
    band, ng = ct.c_int(), ct.c_int()
    st = lib().vmc_lists_layout(lists, ct.byref(band), ct.byref(ng))
    if st != 0:
        raise VmcError(st, "vmc_lists_layout")
    return dict(band=band.value, n_groups=ng.value)


def vmc_lists_near_ties(lists, eps: float) -> int:
    n = ct.c_int64()
    st = lib().vmc_lists_near_ties(lists, float(eps), ct.byref(n))
    if st != 0:
        raise VmcError(st, "vmc_lists_near_ties: eps must be the build eps or above it by more than the band")
    return n.value


def vmc_screened_moves(ctx, lists, params, walkers, eps_run, w_begin, n_w, cap, code, ratio, contrib, count,
                       walked=None):
    if cap > 0:
        _need(code, "code", n_w * cap, _CODES)
        _need(ratio, "ratio", n_w * cap)
        _need(contrib, "contrib", n_w * cap)
    _need(count, "count", n_w, (torch.int64,))
    _need(walked, "walked", 2 * n_w, (torch.int64,))
    _check(ctx, lib().vmc_screened_moves(ctx, lists, ct.byref(params), ct.byref(walkers), float(eps_run),
                                         int(w_begin), int(n_w), int(cap), _ptr(code), _ptr(ratio), _ptr(contrib),
                                         _ptr(count), _ptr(walked)))


def vmc_lists_destroy(lists):
    lib().vmc_lists_destroy(lists)


def vmc_lists_info(lists):
    a, b, c = ct.c_int64(), ct.c_int64(), ct.c_int64()
    _check(None, lib().vmc_lists_info(lists, ct.byref(a), ct.byref(b), ct.byref(c)))
    return a.value, b.value, c.value


def vmc_walkers_sizes(W, M, na, nb, lists):
    out = (ct.c_int64 * 10)()
    _check(None, lib().vmc_walkers_sizes(W, M, na, nb, lists, out))
    return list(out)


def vmc_walkers_init(ctx, lists, params, walkers):
    _check(ctx, lib().vmc_walkers_init(ctx, lists, ct.byref(params), ct.byref(walkers)))


def vmc_walkers_refresh(ctx, lists, params, walkers):
    _check(ctx, lib().vmc_walkers_refresh(ctx, lists, ct.byref(params), ct.byref(walkers)))


def vmc_log_psi(ctx, walkers, params, out):
    _need(out, "out", walkers.W)
    _check(ctx, lib().vmc_log_psi(ctx, ct.byref(walkers), ct.byref(params), _ptr(out)))


def vmc_local_energy(ctx, lists, params, walkers, eps_run, e_loc, t_res):
    _need(e_loc, "e_loc", walkers.W)
    _need(t_res, "t_res", walkers.W)
    _check(ctx, lib().vmc_local_energy(ctx, lists, ct.byref(params), ct.byref(walkers), float(eps_run),
                                       _ptr(e_loc), _ptr(t_res)))


def vmc_ctmc_step(ctx, lists, params, walkers, seed, move_code):
    _need(move_code, "move_code", walkers.W, _CODES)
    _check(ctx, lib().vmc_ctmc_step(ctx, lists, ct.byref(params), ct.byref(walkers), int(seed),
                                    _ptr(move_code)))


def vmc_grad_logpsi(ctx, walkers, w, dJ, dCa, dCb):
    _need(w, "w", walkers.W)
    _need_grad(walkers, dJ, dCa, dCb)
    _check(ctx, lib().vmc_grad_logpsi(ctx, ct.byref(walkers), _ptr(w), _ptr(dJ), _ptr(dCa), _ptr(dCb)))


def vmc_amsgrad_update(ctx, p, g, m, n, alpha, beta1, beta2):
    _need(p, "p", 0)
    for t, name in ((g, "g"), (m, "m"), (n, "n")):
        _need(t, name, p.numel())
    _check(ctx, lib().vmc_amsgrad_update(ctx, _ptr(p), _ptr(g), _ptr(m), _ptr(n), p.numel(),
                                         float(alpha), float(beta1), float(beta2)))


def vmc_walker_reduce(ctx, W, t_res, e_loc, out):
    _need(t_res, "t_res", W)
    _need(e_loc, "e_loc", W)
    _need(out, "out", 2)
    _check(ctx, lib().vmc_walker_reduce(ctx, W, _ptr(t_res), _ptr(e_loc), _ptr(out)))


def vmc_accumulate_gradient(ctx, walkers, t_res, e_loc, AO, AEO, sums):
    """AO, AEO: (dJ, dCa, dCb) tensors each."""
    _need(t_res, "t_res", walkers.W)
    _need(e_loc, "e_loc", walkers.W)
    _need_grad(walkers, *AO, prefix="AO.")
    _need_grad(walkers, *AEO, prefix="AEO.")
    _need(sums, "sums", 2)
    _check(ctx, lib().vmc_accumulate_gradient(ctx, ct.byref(walkers), _ptr(t_res), _ptr(e_loc),
                                              *(_ptr(x) for x in AO), *(_ptr(x) for x in AEO), _ptr(sums)))


def vmc_energy_gradient(ctx, sums, A_O, A_EO, g):
    _need(sums, "sums", 2)
    _need(g, "g", 0)
    _need(A_O, "A_O", g.numel())
    _need(A_EO, "A_EO", g.numel())
    _check(ctx, lib().vmc_energy_gradient(ctx, g.numel(), _ptr(sums), _ptr(A_O), _ptr(A_EO), _ptr(g)))


def vmc_grad_logpsi_noalloc(walkers, w, dJ, dCa, dCb, stream=None):
    """Context-free, allocation-free variant of vmc_grad_logpsi (see include/vmc.h)."""
    _need(w, "w", walkers.W)
    _need_grad(walkers, dJ, dCa, dCb)
    s = stream.cuda_stream if isinstance(stream, torch.cuda.Stream) else (stream or 0)
    st = lib().vmc_grad_logpsi_noalloc(ct.byref(walkers), _ptr(w), _ptr(dJ), _ptr(dCa), _ptr(dCb), s)
    if st != 0:
        raise VmcError(st, "vmc_grad_logpsi_noalloc")


def vmc_local_energy_batch(ctx, items):
    _check(ctx, lib().vmc_local_energy_batch(ctx, len(items), items))


def vmc_ctmc_step_batch(ctx, items, seed):
    _check(ctx, lib().vmc_ctmc_step_batch(ctx, len(items), items, int(seed)))


def vmc_autotune_local_energy(ctx, items) -> int:
    out = ct.c_int()
    _check(ctx, lib().vmc_autotune_local_energy(ctx, len(items), items, ct.byref(out)))
    return out.value


def vmc_set_option(ctx, option: int, value: int):
    _check(ctx, lib().vmc_set_option(ctx, option, value))


def vmc_probe_l2_read(ctx, buf: torch.Tensor, reps: int):
    _need(buf, "buf", 0, (buf.dtype,))
    _check(ctx, lib().vmc_probe_l2_read(ctx, _ptr(buf), buf.numel() * buf.element_size(), int(reps)))


def vmc_cps_create(ctx, M: int, sites) -> ct.c_void_p:
    """Correlator product structure from a list of per-correlator site arrays (see include/vmc.h)."""
    off = np.concatenate([[0], np.cumsum([len(x) for x in sites])]).astype(np.int32)
    flat = np.ascontiguousarray(np.concatenate([np.asarray(x, dtype=np.int32) for x in sites]), dtype=np.int32)
    out = ct.c_void_p()
    _check(ctx, lib().vmc_cps_create(ctx, int(M), len(sites), _ptr(off), _ptr(flat), ct.byref(out)))
    return out


def vmc_cps_destroy(cps):
    lib().vmc_cps_destroy(cps)


def vmc_cps_info(cps):
    n, v = ct.c_int(), ct.c_int64()
    st = lib().vmc_cps_info(cps, ct.byref(n), ct.byref(v))
    if st != 0:
        raise VmcError(st, "vmc_cps_info")
    return n.value, v.value


def vmc_grad_logpsi_cps(ctx, walkers, params, w, dc):
    _need(w, "w", walkers.W)
    _need(dc, "dc", 0)
    _check(ctx, lib().vmc_grad_logpsi_cps(ctx, ct.byref(walkers), ct.byref(params), _ptr(w), _ptr(dc)))


def vmc_accumulate_gradient_cps(ctx, walkers, params, t_res, e_loc, AO_c, AEO_c):
    _need(t_res, "t_res", walkers.W)
    _need(e_loc, "e_loc", walkers.W)
    _need(AO_c, "AO_c", 0)
    _need(AEO_c, "AEO_c", 0)
    _check(ctx, lib().vmc_accumulate_gradient_cps(ctx, ct.byref(walkers), ct.byref(params), _ptr(t_res), _ptr(e_loc),
                                                  _ptr(AO_c), _ptr(AEO_c)))


def vmc_launch_count(ctx) -> int:
    return int(lib().vmc_launch_count(ctx))


# ------------------------------------------------------------------ device buffers
@dataclass
class Walkers:
    """Caller-owned device arrays of the walker state (layout in include/vmc.h)."""
    W: int
    M: int
    n_alpha: int
    n_beta: int
    precision: int
    occ_bits: torch.Tensor
    occ_list: torch.Tensor
    virt_list: torch.Tensor
    pos: torch.Tensor
    G: torch.Tensor
    AinvT: torch.Tensor
    S: torch.Tensor
    F: torch.Tensor
    e_diag: torch.Tensor
    rng_counter: torch.Tensor
    cps_state: torch.Tensor | None = None     # [W][n_corr] int16 (a correlator product only)

    @classmethod
    def allocate(cls, W, M, na, nb, lists, precision=VMC_FP64, device="cuda", n_corr=0):
        n = vmc_walkers_sizes(W, M, na, nb, lists)
        real = torch.float64 if precision == VMC_FP64 else torch.float32
        z = lambda k, dt: torch.zeros(max(1, n[k]), dtype=dt, device=device)
        cps = torch.zeros(W * n_corr, dtype=torch.int16, device=device) if n_corr else None
        return cls(W, M, na, nb, precision, z(0, torch.int32), z(1, torch.int16), z(2, torch.int16),
                   z(3, torch.int16), z(4, real), z(5, real), z(6, real), z(7, real),
                   z(8, torch.float64), z(9, torch.int64), cps)

    def struct(self) -> vmc_walkers:
        return vmc_walkers(self.W, self.M, self.n_alpha, self.n_beta, self.precision,
                           _ptr(self.occ_bits), _ptr(self.occ_list), _ptr(self.virt_list), _ptr(self.pos),
                           _ptr(self.G),
                           _ptr(self.AinvT), _ptr(self.S), _ptr(self.F), _ptr(self.e_diag),
                           _ptr(self.rng_counter), _ptr(self.cps_state))


def params_struct(J: torch.Tensor, Ca: torch.Tensor, Cb: torch.Tensor, cps=None,
                  cps_values: torch.Tensor | None = None) -> vmc_params:
    for t, name in ((J, "J"), (Ca, "C_alpha"), (Cb, "C_beta")):
        _need(t, name, 0)
    if cps is not None:
        _need(cps_values, "cps_values", vmc_cps_info(cps)[1])
    return vmc_params(_ptr(J), _ptr(Ca), _ptr(Cb), cps, _ptr(cps_values))


def decode_moves(codes: np.ndarray) -> np.ndarray:
    """uint64 move codes -> (W, 5) int array (kind, i, j, a, b); j = b = -1 for singles."""
    c = codes.astype(np.uint64)
    out = np.stack([(c & 3), (c >> 2) & 1023, (c >> 12) & 1023, (c >> 22) & 1023, (c >> 32) & 1023],
                   axis=1).astype(np.int64)
    single = out[:, 0] == 1
    out[single, 2] = -1
    out[single, 4] = -1
    return out


class Engine:
    """One Hamiltonian, one parameter set and W walkers on one GPU (thin convenience wrapper)."""

    def __init__(self, system, params, occ: np.ndarray, eps: float, precision: int = VMC_FP64,
                 device: int = 0, stream=None, cps=None):
        """cps: optional correlator product (an object with per-correlator ``sites`` and ``values``
        lists, as systems.CPS); its coefficients follow J, C_alpha, C_beta in the flat parameters."""
        self.device = torch.device("cuda", device)
        self.M, self.na, self.nb = system.M, system.n_alpha, system.n_beta
        self.eps = float(eps)
        self.ctx = vmc_create(device, stream if stream is not None else torch.cuda.current_stream(device))
        self.lists = vmc_build_screened_lists(self.ctx, system.M, system.h1, system.eri, system.e_core, eps)
        self.cps, self.n_corr, self.n_cps = None, 0, 0
        self.cps_sites = None if cps is None else [[int(x) for x in st] for st in cps.sites]
        self.system_name = getattr(system, "name", "")
        parts = [np.asarray(params.J, dtype=np.float64).ravel(), np.asarray(params.C_alpha, dtype=np.float64).ravel(),
                 np.asarray(params.C_beta, dtype=np.float64).ravel()]
        if cps is not None:
            self.cps = vmc_cps_create(self.ctx, system.M, cps.sites)
            self.n_corr, self.n_cps = vmc_cps_info(self.cps)
            parts.append(np.concatenate([np.asarray(v, dtype=np.float64) for v in cps.values]))
            assert parts[-1].size == self.n_cps
        N2 = 2 * self.M
        self.n_params = N2 * N2 + self.M * (self.na + self.nb) + self.n_cps
        self.p = torch.as_tensor(np.concatenate(parts), device=self.device).contiguous()   # one flat buffer
        self.J, self.Ca, self.Cb = self.split(self.p)
        self.c = self.split_cps(self.p)
        self.W = occ.shape[0]
        self.walkers = Walkers.allocate(self.W, self.M, self.na, self.nb, self.lists, precision, self.device,
                                        self.n_corr)
        self.walkers.occ_list.copy_(torch.from_numpy(occ.astype(np.int16).reshape(-1)))
        self.e_loc = torch.zeros(self.W, dtype=torch.float64, device=self.device)
        self.t_res = torch.zeros(self.W, dtype=torch.float64, device=self.device)
        self.moves = torch.zeros(self.W, dtype=torch.int64, device=self.device)
        self.init()

    def split(self, flat: torch.Tensor):
        """Views (J, C_alpha, C_beta) of a flat parameter-shaped buffer."""
        N2 = 2 * self.M
        a = N2 * N2
        b = a + self.M * self.na
        return (flat[:a].view(N2, N2), flat[a:b].view(self.M, self.na),
                flat[b:b + self.M * self.nb].view(self.M, self.nb))

    def split_cps(self, flat: torch.Tensor):
        """View of the correlator coefficients in a flat parameter-shaped buffer (None without them)."""
        if not self.n_cps:
            return None
        a = (2 * self.M) ** 2 + self.M * (self.na + self.nb)
        return flat[a:a + self.n_cps]

    @property
    def params(self) -> vmc_params:
        return params_struct(self.J, self.Ca, self.Cb, self.cps, self.c)

    def init(self):
        vmc_walkers_init(self.ctx, self.lists, self.params, self.walkers.struct())
        self._tables_for = self.p.clone()       # the parameter values the walker tables belong to

    def refresh(self):
        vmc_walkers_refresh(self.ctx, self.lists, self.params, self.walkers.struct())
        self._tables_for = self.p.clone()

    def tables_match(self, J, Ca, Cb) -> bool:
        """True if the walker tables were built for exactly these parameter values."""
        Jt, Cat, Cbt = self.split(self._tables_for)
        return all(x.shape == y.shape and torch.equal(x.detach(), y) for x, y in ((J, Jt), (Ca, Cat), (Cb, Cbt)))

    def local_energy(self, eps_run: float | None = None):
        vmc_local_energy(self.ctx, self.lists, self.params, self.walkers.struct(),
                         self.eps if eps_run is None else eps_run, self.e_loc, self.t_res)
        return self.e_loc, self.t_res

    def ctmc_step(self, seed: int):
        vmc_ctmc_step(self.ctx, self.lists, self.params, self.walkers.struct(), seed, self.moves)
        return self.moves

    def grad_logpsi(self, w: torch.Tensor, dJ=None, dCa=None, dCb=None):
        dJ = torch.zeros_like(self.J) if dJ is None else dJ
        dCa = torch.zeros_like(self.Ca) if dCa is None else dCa
        dCb = torch.zeros_like(self.Cb) if dCb is None else dCb
        vmc_grad_logpsi(self.ctx, self.walkers.struct(), w.contiguous(), dJ, dCa, dCb)
        return dJ, dCa, dCb

    def move_counts(self, eps_run: float | None = None):
        """Per walker: the number of screened moves and the singles and doubles list entries the walk
        reads (vmc_screened_moves with no move buffers), as host arrays (W,) and (W, 2)."""
        eps_run = self.eps if eps_run is None else eps_run
        count = torch.zeros(self.W, dtype=torch.int64, device=self.device)
        walked = torch.zeros(2 * self.W, dtype=torch.int64, device=self.device)
        vmc_screened_moves(self.ctx, self.lists, self.params, self.walkers.struct(), eps_run, 0, self.W, 0,
                           None, None, None, count, walked)
        return count.cpu().numpy(), walked.view(self.W, 2).cpu().numpy()

    def screened_moves(self, w_begin: int = 0, n_w: int | None = None, eps_run: float | None = None,
                       cap: int = 0):
        """The screened move set of walkers [w_begin, w_begin + n_w) (vmc_screened_moves), as
        host arrays: per walker (codes, ratios, contributions) plus the walked entry counts."""
        n_w = self.W - w_begin if n_w is None else n_w
        eps_run = self.eps if eps_run is None else eps_run
        dev = self.device
        count = torch.zeros(n_w, dtype=torch.int64, device=dev)
        walked = torch.zeros(2 * n_w, dtype=torch.int64, device=dev)
        if cap <= 0:   # first pass: the counts size the buffers
            vmc_screened_moves(self.ctx, self.lists, self.params, self.walkers.struct(), eps_run, w_begin, n_w, 0,
                               None, None, None, count, walked)
            cap = max(1, int(count.max().item()))
        code = torch.zeros(n_w * cap, dtype=torch.int64, device=dev)
        ratio = torch.zeros(n_w * cap, dtype=torch.float64, device=dev)
        contrib = torch.zeros(n_w * cap, dtype=torch.float64, device=dev)
        vmc_screened_moves(self.ctx, self.lists, self.params, self.walkers.struct(), eps_run, w_begin, n_w, cap,
                           code, ratio, contrib, count, walked)
        cnt = count.cpu().numpy()
        c, r, e = (x.view(n_w, cap).cpu().numpy() for x in (code, ratio, contrib))
        out = [(c[t, :min(cap, cnt[t])].astype(np.uint64), r[t, :min(cap, cnt[t])], e[t, :min(cap, cnt[t])])
               for t in range(n_w)]
        return out, cnt, walked.view(n_w, 2).cpu().numpy()

    def grad_logpsi_cps(self, w: torch.Tensor, dc=None):
        dc = torch.zeros_like(self.c) if dc is None else dc
        vmc_grad_logpsi_cps(self.ctx, self.walkers.struct(), self.params, w.contiguous(), dc)
        return dc

    def log_psi(self) -> torch.Tensor:
        out = torch.zeros(self.W, dtype=torch.float64, device=self.device)
        vmc_log_psi(self.ctx, self.walkers.struct(), self.params, out)
        return out

    def sync(self):
        vmc_sync(self.ctx)

    def occupations(self) -> np.ndarray:
        """(W, 2M) uint8 occupation numbers from the device bit strings."""
        bits = self.walkers.occ_bits.cpu().numpy().view(np.uint32).reshape(self.W, 2, -1)
        M = self.M
        n = np.zeros((self.W, 2 * M), dtype=np.uint8)
        for s in range(2):
            for k in range(M):
                n[:, s * M + k] = (bits[:, s, k // 32] >> np.uint32(k % 32)) & 1
        return n

    def close(self):
        if getattr(self, "lists", None):
            vmc_lists_destroy(self.lists)
            self.lists = None
        if getattr(self, "cps", None):
            vmc_sync(self.ctx)
            vmc_cps_destroy(self.cps)
            self.cps = None
        if getattr(self, "ctx", None):
            vmc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Several engines (systems of uneven size, same precision) driven by batched launches."""

    def __init__(self, engines):
        self.engines = list(engines)
        self.ctx = self.engines[0].ctx
        self._keep = []
        self.items = (vmc_batch_item * len(self.engines))()
        for k, e in enumerate(self.engines):
            prm = e.params
            ws = e.walkers.struct()
            self._keep += [prm, ws]
            self.items[k] = vmc_batch_item(e.lists, ct.pointer(prm), ct.pointer(ws), e.eps, _ptr(e.e_loc),
                                           _ptr(e.t_res), _ptr(e.moves))

    @property
    def W(self) -> int:
        return sum(e.W for e in self.engines)

    def local_energy(self):
        vmc_local_energy_batch(self.ctx, self.items)

    def ctmc_step(self, seed: int):
        vmc_ctmc_step_batch(self.ctx, self.items, seed)

    def autotune(self) -> int:
        return vmc_autotune_local_energy(self.ctx, self.items)


class LogPsi(torch.autograd.Function):
    """ln|psi(n_w)| per walker as a differentiable function of (J, C_alpha, C_beta).

    forward: vmc_log_psi (FP64 LU per walker); backward: vmc_grad_logpsi, the hand-written
    vector-Jacobian product of the gradient ratios of Sec. III.B.  J enters through its upper
    triangle, so the lower triangle of dJ is zero.

    The backward reads the engine's walker tables (C_occ^-1), so (J, Ca, Cb) must hold the values
    those tables were built for (the engine's parameters at its last init or refresh); any other
    values raise ValueError instead of returning the gradient of different parameters.
    """

    @staticmethod
    def forward(ctx, J, Ca, Cb, engine: Engine):
        if not engine.tables_match(J, Ca, Cb):
            raise ValueError("LogPsi: the walker tables belong to other parameter values; copy these values "
                             "into the engine's parameters and call engine.refresh() first")
        Jc, Cac, Cbc = J.contiguous(), Ca.contiguous(), Cb.contiguous()   # alive until the call is queued
        prm = params_struct(Jc, Cac, Cbc, engine.cps, engine.c)
        out = torch.zeros(engine.W, dtype=torch.float64, device=J.device)
        vmc_log_psi(engine.ctx, engine.walkers.struct(), prm, out)
        ctx.engine = engine
        return out

    @staticmethod
    def backward(ctx, grad_out):
        e = ctx.engine
        dJ, dCa, dCb = e.grad_logpsi(grad_out.contiguous().to(torch.float64))
        return dJ, dCa, dCb, None
