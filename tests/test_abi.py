"""The C-ABI library builds, loads and exports every symbol include/vmc.h declares (CPU only)."""
import ctypes as ct
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


def declared_functions():
    text = (ROOT / "include" / "vmc.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(vmc_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libvmc():
    from paper_1807_10633_gb300 import build
    return ct.CDLL(str(build.build()))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["vmc_build_screened_lists", "vmc_local_energy", "vmc_ctmc_step",
                     "vmc_grad_logpsi", "vmc_amsgrad_update"]:
        assert required in names


def test_every_declared_symbol_is_exported(libvmc):
    missing = [n for n in declared_functions() if not hasattr(libvmc, n)]
    assert not missing, missing


def test_binding_exposes_the_same_names():
    from paper_1807_10633_gb300 import vmc
    for n in declared_functions():
        assert hasattr(vmc, n), n


def test_null_arguments_are_rejected_without_a_gpu(libvmc):
    libvmc.vmc_walkers_sizes.restype = ct.c_int
    out = (ct.c_int64 * 10)()                                              # int64_t out[10]
    assert libvmc.vmc_walkers_sizes(4, 0, 1, 1, None, out) == 1          # M < 1
    assert libvmc.vmc_walkers_sizes(4, 10, 5, 5, None, out) == 0
    assert list(out)[:3] == [4 * 2 * 1, 4 * 10, 4 * 10]
    libvmc.vmc_lists_info.restype = ct.c_int
    assert libvmc.vmc_lists_info(None, None, None, None) == 1


def test_binding_constants_match_the_header():
    """Option numbers, precision and status codes in the binding are the header's values."""
    from paper_1807_10633_gb300 import vmc
    text = re.sub(r"/\*.*?\*/", "", (ROOT / "include" / "vmc.h").read_text(), flags=re.S)
    defines = dict((k, int(v)) for k, v in re.findall(r"#define\s+(VMC_OPT_[A-Z0-9_]+)\s+(\d+)", text))
    enums = dict((k, int(v)) for k, v in re.findall(r"\b(VMC_[A-Z0-9_]+)\s*=\s*(\d+)", text))
    assert defines and enums
    for k, v in defines.items():
        assert getattr(vmc, k) == v, k
    assert (vmc.VMC_FP64, vmc.VMC_MIXED) == (enums["VMC_FP64"], enums["VMC_MIXED"])
    for k, v in enums.items():
        if k.startswith("VMC_ERR_") or k == "VMC_OK":
            assert vmc._STATUS[v] == k[len("VMC_"):], k


def test_noalloc_gradient_rejects_zero_electrons_without_a_gpu(libvmc):
    """With no electron of either spin there is no orbital block to size the scratch by: the call
    must return VMC_ERR_ARG from its host checks (no CUDA call happens before them)."""
    from paper_1807_10633_gb300 import vmc
    fake = 256                                     # never dereferenced: the host check comes first
    ws = vmc.vmc_walkers(8, 4, 0, 0, vmc.VMC_FP64, *([fake] * 10))
    libvmc.vmc_grad_logpsi_noalloc.restype = ct.c_int
    assert libvmc.vmc_grad_logpsi_noalloc(ct.byref(ws), ct.c_void_p(fake), ct.c_void_p(fake),
                                          ct.c_void_p(fake), ct.c_void_p(fake), None) == 1
