"""GPU parity of the event-driven projection (I = bias + sum of the active inputs' weights,
Eq 3 / Prop 3 feedforward term) against the oracle's FP64 product: per output within the
FP32 running-sum bound (k+1) 2^-24 (|bias| + sum_j |W_ij| S_j) for k active inputs, ragged
shapes (N and N_in around the 1024-thread blocks, T not a multiple of 32), dense bursts
that fill a chunk's event list, determinism, and agreement with the tensor-core path."""
import numpy as np
import pytest
import torch

from oracle import project as oproj
from paper_2311_11390_gb300 import synth

pytestmark = pytest.mark.gpu
cuda = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")


def _alif():
    from paper_2311_11390_gb300 import alif
    alif.lib()
    return alif


def _case(seed, B, Nin, N, T, rate_hz=(10.0, 50.0), dt=0.1, burst=False, bias=True):
    rng = np.random.default_rng(seed)
    rates = rng.uniform(*rate_hz, size=Nin)
    S = synth.poisson_raster(rng, B, Nin, T, rates, dt)
    if burst:  # every input fires on a run of steps: full event lists
        S[:, :, 40:72] = True
    W = (rng.standard_normal((N, Nin)) * np.sqrt(2.0 / Nin)).astype(np.float32)
    b = rng.uniform(0.8, 1.6, size=N).astype(np.float32) if bias else None
    return S, W, b


def _run(alif, S, W, b, T):
    words = torch.from_numpy(synth.pack_bits(S).view(np.int32)).cuda()
    Wt = alif.transpose_weights(torch.from_numpy(W).cuda())
    bt = None if b is None else torch.from_numpy(b).cuda()
    I = alif.syn_project_events(words, Wt, bt, Nin=W.shape[1], T=T)
    torch.cuda.synchronize()
    return I.cpu().numpy(), words, Wt, bt


def _check(I, S, W, b):
    ref = oproj.project(W, S, b)
    k = S.sum(axis=1, dtype=np.float64)[:, None, :]  # active inputs per (b, t)
    mag = np.einsum("ij,bjt->bit", np.abs(W.astype(np.float64)), S.astype(np.float64))
    if b is not None:
        mag = mag + np.abs(b.astype(np.float64))[None, :, None]
    bound = (k + 1) * 2.0 ** -24 * mag + 1e-30
    err = np.abs(I.astype(np.float64) - ref)
    assert np.all(err <= bound), f"max err/bound {np.max(err / bound):.3f}"


@cuda
@pytest.mark.parametrize("B, Nin, N, T, burst", [(3, 1000, 200, 1000, False), (2, 2500, 1500, 333, False),
                                                 (2, 1100, 1030, 97, True), (1, 31, 33, 40, True)])
def test_events_match_oracle(B, Nin, N, T, burst):
    alif = _alif()
    S, W, b = _case(B * 7 + T, B, Nin, N, T, burst=burst)
    I, *_ = _run(alif, S, W, b, T)
    _check(I, S, W, b)


@cuda
def test_events_dense_input_and_no_bias():
    """Inputs at 2 kHz (0.2 spikes per 0.1 ms step each): long lists, no bias."""
    alif = _alif()
    S, W, b = _case(5, 2, 700, 256, 500, rate_hz=(1000.0, 3000.0), bias=False)
    I, *_ = _run(alif, S, W, None, 500)
    _check(I, S, W, None)


@cuda
def test_events_deterministic_and_close_to_tensor_core_path():
    alif = _alif()
    S, W, b = _case(9, 4, 1000, 1024, 2048)
    I1, words, Wt, bt = _run(alif, S, W, b, 2048)
    I2 = alif.syn_project_events(words, Wt, bt, Nin=1000, T=2048).cpu().numpy()
    assert np.array_equal(I1, I2)
    hi, lo = alif.split_bf16(torch.from_numpy(W).cuda())
    Itc = alif.syn_project(words, hi, lo, bt, Nin=1000, T=2048).cpu().numpy()
    mag = np.einsum("ij,bjt->bit", np.abs(W.astype(np.float64)), S.astype(np.float64)) + np.abs(b)[None, :, None]
    # split-BF16 bound (2^-16 + (K+2) 2^-24) plus the event path's own (k+1) 2^-24
    assert np.all(np.abs(Itc.astype(np.float64) - I1) <= mag * (2.0 ** -16 + 1100 * 2.0 ** -24) + 1e-6)


@cuda
def test_events_degenerate_shapes():
    alif = _alif()
    dev = "cuda"
    Wt = torch.zeros((5, 7), dtype=torch.float32, device=dev)
    bias = torch.arange(7, dtype=torch.float32, device=dev)
    words = torch.zeros((2, 5, 1), dtype=torch.int32, device=dev)
    I = alif.syn_project_events(words, Wt, bias, Nin=5, T=20)
    assert torch.equal(I, bias[None, :, None].expand(2, 7, 20))
    empty_T = alif.syn_project_events(torch.zeros((2, 5, 0), dtype=torch.int32, device=dev), Wt, bias, Nin=5, T=0)
    assert empty_T.shape == (2, 7, 0)
    no_in = alif.syn_project_events(torch.zeros((2, 0, 1), dtype=torch.int32, device=dev),
                                    torch.zeros((0, 7), dtype=torch.float32, device=dev), bias, Nin=0, T=9)
    assert torch.equal(no_in, bias[None, :, None].expand(2, 7, 9))
