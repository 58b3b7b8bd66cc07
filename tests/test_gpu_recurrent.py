"""GPU parity of the recurrent layer (latency D = T_R, Section 2 / Prop 3) against the oracle's
step-by-step recurrent simulation, and of its detached gradients against the oracle's BPTT on
the oracle's own total current."""
import math

import numpy as np
import pytest
import torch

from oracle import ref
from paper_2311_11390_gb300 import synth
from tests import parity

pytestmark = pytest.mark.gpu
cuda = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")


def _alif():
    from paper_2311_11390_gb300 import alif
    alif.lib()
    return alif


def _case(seed, B, N, T, arp, scale, bias=(1.1, 2.2)):
    w = synth.population(seed=seed, B=B, N=N, T=T, arp=arp, bias=bias, tau_adapt=(60.0, 300.0), d=(0.0, 0.6))
    W = (scale * np.random.default_rng(seed + 7).standard_normal((N, N)) / math.sqrt(N)).astype(np.float32)
    return w, W


def _run(alif, w, W, **kw):
    table = alif.neuron_table(w.params.tau_mem, w.params.tau_adapt, w.params.theta0, w.params.d,
                              w.params.R, w.dt, w.arp)
    Iff = torch.from_numpy(w.I).cuda()
    Wt = alif.transpose_weights(torch.from_numpy(W).cuda())
    out = alif.forward_recurrent(Iff, Wt, table, w.dt, w.arp, **kw)
    torch.cuda.synchronize()
    assert alif.device_status() == 0
    return table, Iff, out


@cuda
@pytest.mark.parametrize("seed, B, N, T, arp, scale", [
    (0, 2, 64, 1000, 2.0, 1.5),      # T_R = 20, one CTA per batch element
    (1, 2, 300, 777, 0.5, 2.0),      # T_R = 5, 3 CTAs per cluster, ragged neurons and Blocks
    (2, 1, 1024, 600, 2.0, -3.0),    # inhibitory, 8 CTAs per cluster
    (3, 2, 96, 900, 0.1, 1.0),       # T_R = 1: spikes exchanged every step
    (4, 1, 200, 1300, 4.0, 2.5),     # T_R = 40
    (7, 1, 256, 1500, 20.0, 2.0),    # T_R = 200: one accumulator, no prefetch of the next Block
    (8, 1, 2048, 450, 10.0, 2.0),    # T_R = 100, 256 neurons per CTA: one accumulator, 16 weights per copy
    (9, 1, 2100, 400, 2.0, 2.0),     # 288 neurons per CTA: the kernel sized for 1024-thread CTAs
])
def test_recurrent_forward_matches_oracle(seed, B, N, T, arp, scale):
    """Spikes equal the oracle's exactly: the kernel carries the current, V and a in
    double-single, so a decision can differ only at margins near 1e-12, and the cases hold
    none within 1e-9 (asserted).  The total current I_ff + W_rec S[t - T_R], rounded to
    FP32, agrees with the oracle's; the blocked feedforward forward on it reproduces spikes
    and checkpoints in every row whose oracle margins stay above 1e-6 (in the others the FP32
    rounding of the current may move a near-tie)."""
    alif = _alif()
    w, W = _case(seed, B, N, T, arp, scale)
    P = parity.oracle_params(w.params)
    o = ref.forward_recurrent(w.I, W, P, w.dt, w.arp, nthreads=4)
    assert np.abs(o.margin).min() > 1e-9
    assert o.S.sum() > 50
    assert not np.array_equal(o.S, ref.forward(w.I, P, w.dt, w.arp).S)   # the coupling matters
    table, Iff, out = _run(alif, w, W)
    S = alif.unpack_spikes(out["spikes"], T).cpu().numpy()
    assert np.array_equal(S, o.S)
    It = out["I_total"].cpu().numpy().astype(np.float64)
    scale_I = np.abs(w.I).max() + np.abs(W).sum(1).max()
    np.testing.assert_allclose(It, o.I_total, rtol=0, atol=4e-7 * scale_I)
    ff = alif.forward(out["I_total"], table)
    torch.cuda.synchronize()
    clear = np.abs(o.margin).min(-1) > 1e-6                              # [B, N] rows without near-ties
    assert clear.mean() > 0.5
    assert np.array_equal(alif.unpack_spikes(ff["spikes"], T).cpu().numpy()[clear], S[clear])
    ck_r, ck_f = out["ckpt"].cpu().numpy()[clear], ff["ckpt"].cpu().numpy()[clear]
    assert np.array_equal(ck_r[..., 2], ck_f[..., 2])                    # rem
    np.testing.assert_allclose(ck_r[..., :2].view(np.float32), ck_f[..., :2].view(np.float32),
                               rtol=1e-6, atol=1e-6)                     # v, a


@cuda
def test_recurrent_in_place_and_final_state():
    """I_total written over I_ff (in place) gives the same spikes and current as a separate
    output, and the final state has the alif_forward layout."""
    alif = _alif()
    w, W = _case(5, 2, 128, 800, 2.0, 1.5)
    table, Iff, out = _run(alif, w, W)
    I2 = Iff.clone()
    out2 = alif.forward_recurrent(I2, alif.transpose_weights(torch.from_numpy(W).cuda()), table, w.dt, w.arp,
                                  in_place=True)
    torch.cuda.synchronize()
    assert torch.equal(out2["spikes"], out["spikes"]) and torch.equal(I2, out["I_total"])
    fin = out["final"].cpu().numpy()
    assert fin.shape == (2, 128, 3)


@cuda
@pytest.mark.parametrize("T, D", [(100, 0), (100, 1), (333, 5), (333, 31), (333, 32), (333, 33), (1000, 100),
                                  (70, 75)])
def test_delay_spikes_bit_exact(T, D):
    alif = _alif()
    rng = np.random.default_rng(T + D)
    S = (rng.random((3, 5, T)) < 0.3).astype(np.uint8)
    words = alif.pack_spikes(torch.from_numpy(S.astype(np.float32)).cuda())
    out = alif.delay_spikes(words, T, D)
    got = alif.unpack_spikes(out, T).cpu().numpy()
    want = np.zeros_like(S)
    if D < T:
        want[..., D:] = S[..., :T - D]
    assert np.array_equal(got, want)


@cuda
def test_recurrent_backward_matches_oracle():
    """Detached gradients of the recurrent layer: the recurrent synapses carry no gradient into
    S, so dL/dI and the neuron parameters' gradients are the block backward on the total
    current, and dL/dW_rec = sum_t dL/dI[t] S[t - T_R]^T.  Against the oracle's BPTT on its own
    total current and the same sum over its own spikes, in float64."""
    alif = _alif()
    w, W = _case(6, 2, 160, 1100, 2.0, 2.0)
    P = parity.oracle_params(w.params)
    o = ref.forward_recurrent(w.I, W, P, w.dt, w.arp, nthreads=4)
    assert np.abs(o.margin).min() > 1e-9
    table, Iff, out = _run(alif, w, W)
    S = alif.unpack_spikes(out["spikes"], w.I.shape[-1]).cpu().numpy()
    assert np.array_equal(S, o.S)
    rng = np.random.default_rng(6)
    gS = rng.standard_normal(w.I.shape)
    gI, _, gp = alif.backward(out["I_total"], table, out["spikes"], torch.from_numpy(gS.astype(np.float32)).cuda(),
                              ckpt=out["ckpt"])
    TR = alif.tr(w.dt, w.arp)
    gW, _, _ = alif.syn_project_backward(alif.delay_spikes(out["spikes"], w.I.shape[-1], TR), gI, Nin=W.shape[0],
                                         want_gb=False)
    torch.cuda.synchronize()
    ob = ref.backward(o.I_total.astype(np.float32), P, w.dt, w.arp, gS)
    parity.grad_close(gI.cpu().numpy(), ob.gI, what="grad_I")
    for k, n in enumerate(["g_tau_mem", "g_tau_adapt", "g_theta0", "g_d", "g_R"]):
        parity.grad_close(gp[k].cpu().numpy(), getattr(ob, n).sum(0), what=n)
    Sd = np.zeros_like(o.S, np.float64)
    Sd[..., TR:] = o.S[..., :-TR]
    gW_o = np.einsum("bit,bjt->ij", ob.gI, Sd)
    parity.grad_close(gW.cpu().numpy(), gW_o, what="grad_W_rec")
