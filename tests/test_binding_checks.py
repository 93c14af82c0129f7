"""The binding rejects device-tensor arguments whose dtype, size or device would let a kernel read
or write past a buffer, before anything crosses the ABI (CPU only: no call reaches the library)."""
import pytest
import torch

from paper_1807_10633_gb300 import vmc

W, M, NA, NB = 8, 4, 2, 1
F64 = torch.float64


@pytest.fixture
def ws():
    return vmc.vmc_walkers(W, M, NA, NB, vmc.VMC_FP64, *([None] * 10))


def test_local_energy_outputs(ws):
    ok = torch.zeros(W, dtype=F64)
    with pytest.raises(ValueError, match="dtype"):
        vmc.vmc_local_energy(None, None, vmc.vmc_params(), ws, 1e-6, torch.zeros(W, dtype=torch.float32), ok)
    with pytest.raises(ValueError, match="at least 8"):
        vmc.vmc_local_energy(None, None, vmc.vmc_params(), ws, 1e-6, torch.zeros(W - 1, dtype=F64), ok)
    with pytest.raises(ValueError, match="CUDA"):
        vmc.vmc_local_energy(None, None, vmc.vmc_params(), ws, 1e-6, ok, ok)
    with pytest.raises(TypeError):
        vmc.vmc_local_energy(None, None, vmc.vmc_params(), ws, 1e-6, [0.0] * W, ok)


def test_move_codes_are_64_bit_integers(ws):
    with pytest.raises(ValueError, match="dtype"):
        vmc.vmc_ctmc_step(None, None, vmc.vmc_params(), ws, 1, torch.zeros(W, dtype=F64))
    with pytest.raises(ValueError, match="at least 8"):
        vmc.vmc_ctmc_step(None, None, vmc.vmc_params(), ws, 1, torch.zeros(W - 1, dtype=torch.int64))


def test_gradient_outputs_have_parameter_shapes(ws):
    w = torch.zeros(W, dtype=F64)
    dJ, dCa, dCb = torch.zeros(4 * M * M, dtype=F64), torch.zeros(M * NA, dtype=F64), torch.zeros(M * NB, dtype=F64)
    # the first argument checked is the faulty one (a CPU tensor that passes would fail as "CUDA")
    with pytest.raises(ValueError, match="w:"):
        vmc.vmc_grad_logpsi(None, ws, w[:-1], dJ, dCa, dCb)
    with pytest.raises(ValueError, match="w: must be a CUDA"):
        vmc.vmc_grad_logpsi_noalloc(ws, w, dJ, dCa, dCb[:-1])
    with pytest.raises(ValueError, match="t_res"):
        vmc.vmc_accumulate_gradient(None, ws, w.float(), w, (dJ, dCa, dCb), (dJ, dCa, dCb), w[:2])


def test_optimizer_vectors_match_the_parameters():
    p = torch.zeros(10, dtype=F64)
    with pytest.raises(ValueError, match="p: must be a CUDA"):
        vmc.vmc_amsgrad_update(None, p, p, p[:9], p, 0.01, 0.1, 0.01)
    with pytest.raises(ValueError, match="sums: 1 elements"):
        vmc.vmc_energy_gradient(None, torch.zeros(1, dtype=F64), p, p[:5], p)
    with pytest.raises(ValueError, match="t_res: 3 elements"):
        vmc.vmc_walker_reduce(None, 4, p[:3], p, torch.zeros(1, dtype=F64))


def test_parameters_must_be_fp64_device_tensors():
    J = torch.zeros(4 * M * M, dtype=F64)
    with pytest.raises(ValueError, match="J: dtype"):
        vmc.params_struct(J.float(), torch.zeros(M * NA, dtype=F64), torch.zeros(M * NB, dtype=F64))
    with pytest.raises(ValueError, match="J: must be a CUDA"):
        vmc.params_struct(J, torch.zeros(M * NA, dtype=F64), torch.zeros(M * NB, dtype=F64))


def test_gradient_block_sizes_follow_the_walker_shapes(ws):
    dJ, dCa, dCb = torch.zeros(4 * M * M, dtype=F64), torch.zeros(M * NA, dtype=F64), torch.zeros(M * NB, dtype=F64)
    with pytest.raises(ValueError, match="dJ: 63 elements, at least 64"):
        vmc._need_grad(ws, dJ[:-1], dCa, dCb)
    with pytest.raises(ValueError, match="AEO.dC_beta: 3 elements, at least 4"):
        vmc._need_grad(ws, None, None, dCb[:-1], prefix="AEO.")      # None: an absent optional output
