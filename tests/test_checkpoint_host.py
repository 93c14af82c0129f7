"""Checkpoint file format on the CPU (no library call): what `save` writes `read` returns unchanged,
a checkpoint of another system or format is refused, and the flat parameters split back into the
pair Jastrow, both Slater blocks and the correlators in the order the engine concatenates them."""
from types import SimpleNamespace

import numpy as np
import pytest
import torch

from paper_1807_10633_gb300 import checkpoint as C
from paper_1807_10633_gb300 import systems as S
from paper_1807_10633_gb300 import vmc
from paper_1807_10633_gb300.optimize import OptState


def _fake_engine(sys_, W, cps=None, precision=vmc.VMC_MIXED, seed=0):
    """An object with the engine attributes `save` reads, filled with seeded values on the CPU."""
    rng = np.random.default_rng(seed)
    M, na, nb = sys_.M, sys_.n_alpha, sys_.n_beta
    prm = S.make_params(sys_, seed=seed)
    parts = [prm.flat()] + ([np.concatenate(cps.values)] if cps else [])
    p = torch.from_numpy(np.concatenate(parts))
    occ = S.init_occupations(sys_, prm, W, seed=seed + 1)
    real = np.float64 if precision == vmc.VMC_FP64 else np.float32
    walkers = SimpleNamespace(precision=precision, occ_list=torch.from_numpy(occ.astype(np.int16).reshape(-1)),
                              rng_counter=torch.from_numpy(rng.integers(0, 1000, W).astype(np.int64)),
                              e_diag=torch.from_numpy(rng.normal(size=W)),
                              F=torch.from_numpy(rng.normal(size=2 * W * 12).astype(real)))
    return SimpleNamespace(M=M, na=na, nb=nb, W=W, eps=1e-6, p=p, walkers=walkers,
                           cps_sites=None if cps is None else [list(s) for s in cps.sites]), prm


@pytest.mark.parametrize("with_cps", [False, True])
def test_save_read_round_trip(tmp_path, with_cps):
    sys_ = S.named_system("H6")
    cps = S.make_cps(sys_, seed=3) if with_cps else None
    eng, prm = _fake_engine(sys_, 17, cps)
    st = OptState(torch.linspace(-1, 1, eng.p.numel(), dtype=torch.float64),
                  torch.linspace(0, 2, eng.p.numel(), dtype=torch.float64), 11)
    path = C.save(tmp_path / "ck", eng, st, sys_)
    assert path.name == "ck"
    ck = C.read(path, sys_)
    np.testing.assert_array_equal(ck["p"], eng.p.numpy())
    np.testing.assert_array_equal(ck["m"], st.m.numpy())
    np.testing.assert_array_equal(ck["v"], st.v.numpy())
    assert int(ck["next_iter"]) == 11 and float(ck["eps"]) == 1e-6
    np.testing.assert_array_equal(ck["occ_list"].ravel(), eng.walkers.occ_list.numpy())
    for k in ("rng_counter", "e_diag", "F"):
        np.testing.assert_array_equal(ck[k], getattr(eng.walkers, k).numpy())
        assert ck[k].dtype == getattr(eng.walkers, k).numpy().dtype
    prm2, cps2 = C.wavefunction(ck)
    np.testing.assert_array_equal(prm2.J, prm.J)
    np.testing.assert_array_equal(prm2.C_alpha, prm.C_alpha)
    np.testing.assert_array_equal(prm2.C_beta, prm.C_beta)
    if with_cps:
        assert cps2.sites == [list(s) for s in cps.sites]
        for a, b in zip(cps2.values, cps.values):
            np.testing.assert_array_equal(a, b)
    else:
        assert cps2 is None


def test_read_refuses_another_system_or_format(tmp_path):
    sys_ = S.named_system("H6")
    eng, _ = _fake_engine(sys_, 5)
    st = OptState(torch.zeros(eng.p.numel(), dtype=torch.float64), torch.zeros(eng.p.numel(), dtype=torch.float64))
    path = C.save(tmp_path / "ck.npz", eng, st, sys_)
    other = S.hchain(6, spacing=1.9)
    with pytest.raises(ValueError, match="different system"):
        C.read(path, other)
    with pytest.raises(ValueError):
        C.save(tmp_path / "x.npz", eng, st, S.named_system("H4"))
    with np.load(path) as z:
        bad = {k: z[k] for k in z.files}
    bad["format"] = np.array(C.FORMAT + 1)
    with open(tmp_path / "bad.npz", "wb") as f:
        np.savez(f, **bad)
    with pytest.raises(ValueError, match="format"):
        C.read(tmp_path / "bad.npz", sys_)


def test_optimisation_cli_resume_checks_the_system_first(tmp_path):
    """`python -m paper_1807_10633_gb300.optimize --resume FILE` refuses a checkpoint of another
    system before any device work; the checkpoint options parse as documented."""
    from paper_1807_10633_gb300 import optimize as O
    sys_ = S.named_system("H6")
    eng, _ = _fake_engine(sys_, 4)
    st = OptState(torch.zeros(eng.p.numel(), dtype=torch.float64), torch.zeros(eng.p.numel(), dtype=torch.float64))
    path = C.save(tmp_path / "h6.ckpt", eng, st, sys_)
    with pytest.raises(ValueError, match="different system"):
        O.main(["--system", "H4", "--resume", str(path)])
    a = O.parser().parse_args(["--iters", "7", "--checkpoint", "run.ckpt", "--checkpoint-every", "3"])
    assert (a.iters, a.checkpoint, a.checkpoint_every, a.resume) == (7, "run.ckpt", 3, "")
