"""GPU parity of the split-BF16 tcgen05 projection against the FP64 projection oracle."""
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


def _bound(W, S, bias, K):
    """Per output: sum_j |W_ij| S_j (2^-16 + (K + 2) 2^-24) + 2^-23 |I*| (split error of
    each weight, FP32 accumulation of K terms, final bias add)."""
    absW = np.abs(W.astype(np.float64))
    mag = np.einsum("ij,bjt->bit", absW, S.astype(np.float64))
    ref = project.project(W, S, bias)
    return mag * (2.0 ** -16 + (K + 2) * 2.0 ** -24) + 2.0 ** -23 * np.abs(ref) + 1e-30, ref


def _run(alif, W, S, bias):
    Wd = torch.from_numpy(W).cuda()
    hi, lo = alif.split_bf16(Wd)
    Sw = torch.from_numpy(synth.pack_bits(S).view(np.int32)).cuda()
    bd = None if bias is None else torch.from_numpy(bias).cuda()
    out = alif.syn_project(Sw, hi, lo, bd, Nin=S.shape[1], T=S.shape[2])
    torch.cuda.synchronize()
    assert alif.device_status() == 0
    return out.cpu().numpy(), hi, lo


@cuda
def test_split_matches_definition():
    alif = _alif()
    rng = np.random.default_rng(0)
    W = (rng.standard_normal((300, 1000)) * np.sqrt(2 / 1000)).astype(np.float32)
    hi, lo = alif.split_bf16(torch.from_numpy(W).cuda())
    hi, lo = hi.cpu().numpy().view(np.uint16), lo.cpu().numpy().view(np.uint16)
    assert hi.shape == (300, 1024)
    rh, rl = project.split_bf16(W)
    as_bits = lambda x: (x.view(np.uint32) >> 16).astype(np.uint16)
    assert np.array_equal(hi[:, :1000], as_bits(rh)) and np.array_equal(lo[:, :1000], as_bits(rl))
    assert np.all(hi[:, 1000:] == 0) and np.all(lo[:, 1000:] == 0)


@cuda
@pytest.mark.parametrize("B, Nin, N, T, p", [(2, 100, 200, 300, 0.2), (1, 64, 128, 256, 0.5),
                                             (2, 700, 256, 1000, 0.02), (3, 1000, 1024, 517, 0.003),
                                             (1, 7, 5, 33, 0.5)])
def test_projection_within_split_bound(B, Nin, N, T, p):
    alif = _alif()
    rng = np.random.default_rng(B * 1000 + Nin)
    W = (rng.standard_normal((N, Nin)) * np.sqrt(2 / Nin)).astype(np.float32)
    S = rng.random((B, Nin, T)) < p
    bias = rng.uniform(0.8, 1.6, N).astype(np.float32)
    out, _, _ = _run(alif, W, S, bias)
    lim, ref = _bound(W, S, bias, Nin)
    err = np.abs(out.astype(np.float64) - ref)
    worst = np.unravel_index(np.argmax(err / lim), err.shape)
    assert np.all(err <= lim), f"worst {worst}: err {err[worst]:.3e} > bound {lim[worst]:.3e}"


@cuda
def test_projection_exact_for_bf16_weights():
    """Weights representable in BF16: lo = 0, every product exact, only FP32 accumulation rounds."""
    alif = _alif()
    rng = np.random.default_rng(5)
    B, Nin, N, T = 2, 192, 256, 512
    W = project.bf16_round((rng.standard_normal((N, Nin)) * 0.1).astype(np.float32))
    S = rng.random((B, Nin, T)) < 0.1
    out, _, lo = _run(alif, W, S, None)
    assert int(lo.abs().max()) == 0
    ref = project.project(W, S)
    mag = np.einsum("ij,bjt->bit", np.abs(W.astype(np.float64)), S.astype(np.float64))
    assert np.all(np.abs(out - ref) <= (Nin + 1) * 2.0 ** -24 * mag + 1e-30)
    # integer-valued weights and few active inputs: the FP32 sum is exact
    Wi = rng.integers(-8, 9, size=(N, Nin)).astype(np.float32)
    out_i, _, _ = _run(alif, Wi, S, None)
    assert np.array_equal(out_i, project.project(Wi, S).astype(np.float32))


@cuda
def test_projection_no_inputs_and_errors():
    alif = _alif()
    bias = torch.arange(4, dtype=torch.float32, device="cuda")
    S = torch.zeros((2, 0, 3), dtype=torch.int32, device="cuda")
    hi = torch.zeros((4, 64), dtype=torch.int16, device="cuda")
    out = alif.syn_project(S, hi, hi, bias, Nin=0, T=70)
    assert torch.equal(out, bias[None, :, None].expand(2, 4, 70))
    bad = torch.zeros((4, 100), dtype=torch.int16, device="cuda")
    with pytest.raises(alif.AlifError):
        alif.syn_project(torch.zeros((1, 100, 2), dtype=torch.int32, device="cuda"), bad, bad, None, T=64)
