"""Walker-table refresh (Sec. III.B): the register-resident Gauss-Jordan inverse (FP64 form; FP32
option of the mixed form) against an FP64 inverse of C_occ computed here, and against the
shared-memory kernels (the mixed form's default FP64 LU), for every tile size the register kernel is
built for (n_sigma up to 16, 64, 80, 96 and 128).  The FP64 form's G from exact digit products on
the tensor cores is checked against G from FP64 FMAs on the CUDA cores, including more than one
tile of 80 virtual orbitals and n_sigma = 128."""
import numpy as np
import pytest
import torch

from paper_1807_10633_gb300 import systems as S

pytestmark = pytest.mark.gpu

# (ring sites, n_alpha, n_beta): register tiles R = ceil(n_max / 16) in {1, 3, 5, 6, 7}
CASES = [(20, 10, 9), (60, 40, 30), (90, 80, 75), (96, 90, 85), (98, 97, 64), (120, 30, 25), (136, 128, 120)]


@pytest.fixture(scope="module")
def vmc():
    from paper_1807_10633_gb300 import vmc as v
    v.lib()
    return v


def _tables(eng):
    eng.sync()
    wk = eng.walkers
    return {k: getattr(wk, k).cpu().numpy().copy() for k in ("G", "AinvT", "occ_bits", "virt_list", "pos", "S")}


def _expected(sys_, prm, occ):
    """G (virtual rows, ascending orbital) and C_occ^-T per walker and spin, in FP64."""
    M, na, nb = sys_.M, sys_.n_alpha, sys_.n_beta
    G, A = [], []
    for w in range(occ.shape[0]):
        for s, C, n, o in ((0, prm.C_alpha, na, occ[w, :na]), (1, prm.C_beta, nb, occ[w, na:])):
            if n == 0:
                continue
            v = np.setdiff1d(np.arange(M), o.astype(np.int64))
            inv = np.linalg.inv(C[o.astype(np.int64)])          # C_occ^-1
            G.append((C[v] @ inv).ravel())
            A.append(inv.T.ravel())                              # AinvT[c][x] = (C_occ^-1)[x][c]
    return np.concatenate(G), np.concatenate(A)


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"M{c[0]}_n{c[1]}_{c[2]}")
@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_register_refresh(vmc, case, precision):
    M, na, nb = case
    sys_ = S.hubbard(M, n_alpha=na, n_beta=nb)
    prm = S.make_params(sys_, seed=11)
    occ = S.init_occupations(sys_, prm, 37, seed=12)
    eng = vmc.Engine(sys_, prm, occ, eps=1e-6, precision=precision)
    try:
        if precision == 1:   # the mixed form's register kernel is the FP32 Gauss-Jordan option
            vmc.vmc_set_option(eng.ctx, vmc.VMC_OPT_MIXED_REFRESH_GJ32, 1)
            eng.refresh()
        reg = _tables(eng)
        G, A = _expected(sys_, prm, occ)
        scale = max(1.0, np.abs(G).max())
        tol = 1e-10 if precision == 0 else 2e-4
        assert np.abs(reg["G"][:G.size] - G).max() / scale < tol
        assert np.abs(reg["AinvT"][:A.size] - A).max() / max(1.0, np.abs(A).max()) < tol
        if max(na, nb) <= 118:                                   # the shared-memory kernels' limit
            for tc in ([0, 1] if precision == 1 else [1]):
                vmc.vmc_set_option(eng.ctx, vmc.VMC_OPT_G_TENSOR_CORES, tc)
                if precision == 1:   # the mixed default: FP64 LU in shared memory
                    vmc.vmc_set_option(eng.ctx, vmc.VMC_OPT_MIXED_REFRESH_GJ32, 0)
                else:
                    vmc.vmc_set_option(eng.ctx, vmc.VMC_OPT_REFRESH_SMEM, 1)
                eng.refresh()
                ref = _tables(eng)
                vmc.vmc_set_option(eng.ctx, vmc.VMC_OPT_REFRESH_SMEM, 0)
                if precision == 1:
                    vmc.vmc_set_option(eng.ctx, vmc.VMC_OPT_MIXED_REFRESH_GJ32, 1)
                    assert np.abs(ref["AinvT"][:A.size] - A).max() / max(1.0, np.abs(A).max()) < tol
                for k in ("occ_bits", "virt_list", "pos", "S"):
                    assert np.array_equal(reg[k], ref[k]), k
                assert np.abs(ref["G"] - reg["G"]).max() / scale < 2 * tol
    finally:
        eng.close()


# (system, walkers): virtual orbitals per spin 10, 80 (one full tile), 90/95 (two tiles), 8/16,
# 179/181 (three tiles, odd n_sigma)
G_CASES = [("H20", 64), ("ring160_80_80", 24), ("ring120_30_25", 40), ("ring136_128_120", 16), ("ring200_21_19", 8)]


def _g_system(name):
    if name.startswith("ring"):
        M, na, nb = (int(x) for x in name[4:].split("_"))
        return S.hubbard(M, n_alpha=na, n_beta=nb)
    return S.named_system(name)


def _row_scale_exponents(X):
    """E per row with |x| < 2^E for every element (frexp's exponent of the largest |x|)."""
    return np.frexp(np.abs(X).max(axis=1))[1]


def _digit_bound(sys_, prm, tables, W):
    """Per element of G: n 2^-42 2^(E_c + F_k), E_c of row c of C_occ^-T, F_k of orbital row k of C
    (the digit-product error bound is about n 2^-43 of that scale)."""
    M, na, nb = sys_.M, sys_.n_alpha, sys_.n_beta
    A, V = tables["AinvT"], tables["virt_list"].astype(np.int64)
    out, ao, vo = [], 0, 0
    for w in range(W):
        for C, n in ((prm.C_alpha, na), (prm.C_beta, nb)):
            nv = M - n
            if n == 0 or nv == 0:
                vo += nv
                ao += n * n
                continue
            Ec = _row_scale_exponents(A[ao:ao + n * n].reshape(n, n))
            Fk = _row_scale_exponents(C[V[vo:vo + nv]])
            out.append((n * np.ldexp(1.0, -42) * np.ldexp(1.0, Fk[:, None] + Ec[None, :])).ravel())
            ao += n * n
            vo += nv
    return np.concatenate(out)


@pytest.mark.parametrize("case", G_CASES, ids=lambda c: c[0])
def test_fp64_g_digit_products(vmc, case):
    """G = C_v C_occ^-1 in the FP64 form: six BF16 digits per operand row on tcgen05 against FP64
    FMAs (G_TENSOR_CORES = 0), every element within n 2^-42 of its two rows' power-of-two scales
    (the bound of the dropped digit products, with a margin of two); E_L within 1e-11 relative."""
    name, W = case
    sys_ = _g_system(name)
    prm = S.make_params(sys_, seed=21)
    occ = S.init_occupations(sys_, prm, W, seed=22)
    eng = vmc.Engine(sys_, prm, occ, eps=1e-6, precision=0)
    try:
        tc = _tables(eng)
        e_tc, _ = eng.local_energy()
        e_tc = e_tc.cpu().numpy().copy()
        vmc.vmc_set_option(eng.ctx, vmc.VMC_OPT_G_TENSOR_CORES, 0)
        eng.refresh()
        cc = _tables(eng)
        e_cc, _ = eng.local_energy()
        e_cc = e_cc.cpu().numpy()
        for k in ("AinvT", "occ_bits", "virt_list", "pos", "S"):
            assert np.array_equal(tc[k], cc[k]), k
        bound = _digit_bound(sys_, prm, cc, W)
        err = np.abs(tc["G"][:bound.size] - cc["G"][:bound.size])
        assert np.all(err <= bound), float((err / bound).max())
        assert np.abs(e_tc - e_cc).max() / max(1.0, np.abs(e_cc).max()) < 1e-11
    finally:
        eng.close()
