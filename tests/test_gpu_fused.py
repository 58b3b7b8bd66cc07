"""The projection fused into the block forward (alif_forward_fused): currents computed in the
forward from the input events against the FP64 projection, spikes against the FP64 oracle on
those currents, and every output bitwise equal to alif_forward() run on the same currents."""
import numpy as np
import pytest
import torch

from oracle import project
from paper_2311_11390_gb300 import synth
from tests import parity

pytestmark = pytest.mark.gpu
cuda = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")


def _alif():
    from paper_2311_11390_gb300 import alif
    alif.lib()
    return alif


@cuda
@pytest.mark.parametrize("B, Nin, N, T, rates", [(2, 1000, 96, 1000, (10.0, 50.0)), (3, 300, 40, 1001, (40.0, 200.0)),
                                                 (1, 1024, 33, 3000, (5.0, 20.0)), (2, 7, 64, 515, (100.0, 300.0))])
def test_fused_forward_matches_projection_and_oracle(B, Nin, N, T, rates):
    alif = _alif()
    w = synth.feedforward(seed=Nin + T, B=B, Nin=Nin, N=N, T=T, rates=rates)
    dev = torch.device("cuda")
    table = alif.neuron_table(w.params.tau_mem, w.params.tau_adapt, w.params.theta0, w.params.d, w.params.R,
                              w.dt, w.arp, device=dev)
    S = torch.from_numpy(synth.pack_bits(w.S_in).view(np.int32)).to(dev)
    W = torch.from_numpy(w.W).to(dev)
    bias = torch.from_numpy(w.bias).to(dev)
    out = alif.forward_fused(S, W, bias, table, T, max_events_per_word=1024)
    torch.cuda.synchronize()
    assert alif.device_status() == 0
    I = out["I"].cpu().numpy()
    # currents: the exact FP32 weights summed in order, within (k+1) 2^-24 (|b| + sum |W| S) of FP64
    ref = project.project(w.W, w.S_in, w.bias)
    k = w.S_in.sum(1, keepdims=True).astype(np.float64)
    mag = np.abs(w.bias.astype(np.float64))[None, :, None] + np.einsum(
        "ij,bjt->bit", np.abs(w.W.astype(np.float64)), w.S_in.astype(np.float64))
    assert np.all(np.abs(I - ref) <= (k + 1) * 2.0 ** -24 * mag + 1e-30)
    # the forward on those currents: spikes as the oracle's, outputs as alif_forward's, bit for bit
    plain = alif.forward(out["I"], table)
    torch.cuda.synchronize()
    for key in ("spikes", "ckpt", "final"):
        assert torch.equal(out[key], plain[key]), key
    Sg = alif.unpack_spikes(out["spikes"], T).cpu().numpy()
    res = parity.compare_forward(Sg, None, None, I, w.params, w.dt, w.arp)
    parity.assert_forward_parity(res)
    assert res["spikes"] > 0


@cuda
def test_fused_forward_reports_bucket_overflow():
    """More active inputs in a 32-step word than the bucket holds: the call completes and the
    device status says ALIF_EUNSUPPORTED (no fault, no partial result presented as valid)."""
    alif = _alif()
    w = synth.feedforward(seed=1, B=1, Nin=256, N=32, T=256, rates=(400.0, 600.0))
    dev = torch.device("cuda")
    table = alif.neuron_table(w.params.tau_mem, w.params.tau_adapt, w.params.theta0, w.params.d, w.params.R,
                              w.dt, w.arp, device=dev)
    S = torch.from_numpy(synth.pack_bits(w.S_in).view(np.int32)).to(dev)
    alif.forward_fused(S, torch.from_numpy(w.W).to(dev), None, table, 256, max_events_per_word=4)
    assert alif.device_status() == -4
    assert alif.device_status() == 0  # cleared by the read
