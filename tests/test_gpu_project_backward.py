"""GPU parity of the projection backward (grad_W, grad_bias event-driven; grad_S on the tcgen05
tensor cores) and of
the spike unpacking kernel, against the FP64 oracle definitions."""
import numpy as np
import pytest
import torch

from oracle import project
from paper_2311_11390_gb300 import synth

pytestmark = pytest.mark.gpu
cuda = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")


def _alif():
    from paper_2311_11390_gb300 import alif
    alif.lib()
    return alif


@cuda
@pytest.mark.parametrize("B, Nin, N, T, p", [(2, 100, 70, 300, 0.05), (3, 700, 256, 1000, 0.02),
                                             (1, 1500, 40, 65, 0.3), (2, 33, 129, 31, 0.5),
                                             (2, 1100, 50, 2333, 0.01)])
def test_projection_backward(B, Nin, N, T, p):
    alif = _alif()
    rng = np.random.default_rng(Nin + T)
    W = (rng.standard_normal((N, Nin)) * 0.05).astype(np.float32)
    S = rng.random((B, Nin, T)) < p
    gI = rng.standard_normal((B, N, T)).astype(np.float32)
    Sw = torch.from_numpy(synth.pack_bits(S).view(np.int32)).cuda()
    gW, gS, gb = alif.syn_project_backward(Sw, torch.from_numpy(gI).cuda(), W=torch.from_numpy(W).cuda(),
                                           Nin=Nin, want_gS=True)
    torch.cuda.synchronize()
    rW, rS, rb = project.project_backward(W, S, gI)
    g64 = np.abs(gI.astype(np.float64))
    # FP32 summation bounds: (#additions) 2^-24 sum |terms|
    magW = np.einsum("bit,bjt->ij", g64, S.astype(np.float64))
    assert np.all(np.abs(gW.cpu().numpy() - rW) <= (T // 32 + B + 34) * 2.0 ** -24 * magW + 1e-30)
    assert np.all(np.abs(gb.cpu().numpy() - rb) <= (T + B + 2) * 2.0 ** -24 * g64.sum((0, 2)) + 1e-30)
    # grad_S on the tensor cores: W and grad_I each split into two BF16 terms (residual <= 2^-16
    # of the value), three exact products per term, FP32 accumulation of 3N products
    magS = np.einsum("ij,bit->bjt", np.abs(W.astype(np.float64)), g64)
    err = np.abs(gS.cpu().numpy() - rS)
    assert np.all(err <= (3 * 2.0 ** -16 + (3 * N + 2) * 2.0 ** -24) * magS + 1e-30)
    # and in practice far inside it: relative L2 error of the whole tensor
    assert np.linalg.norm(err) <= 2e-5 * np.linalg.norm(rS)


@cuda
@pytest.mark.parametrize("T", [1, 32, 77, 1024, 1025, 3000])
def test_unpack_spikes_matches_definition(T):
    """Bits -> float 0/1, one warp per (row, 1024-step chunk): partial words, exact chunk
    multiples and several chunks per row."""
    alif = _alif()
    rng = np.random.default_rng(T)
    S = rng.random((3, 5, T)) < 0.3
    w = torch.from_numpy(synth.pack_bits(S).view(np.int32)).cuda()
    out = alif.spikes_to_float(w, T).cpu().numpy()
    assert np.array_equal(out, S.astype(np.float32))
