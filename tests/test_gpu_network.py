"""GPU parity of the classification network (projection -> ALIF -> projection -> ALIF ->
leaky readout -> cross-entropy, trained through torch.autograd) against the oracle composed
layer by layer: every oracle stage takes the GPU's inputs to that stage (the previous layer's
spikes, which are exact bits, and the GPU's FP32 currents), so each stage is checked at its
own tolerance and the gradients are the oracle's FP64 reverse chain through the same spikes."""
import numpy as np
import pytest
import torch

from oracle import network as onet
from oracle import project as oproj
from oracle import ref
from paper_2311_11390_gb300 import synth
from tests import parity

pytestmark = pytest.mark.gpu
cuda = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")


def _run(seed, B, T, dt, hidden=(48, 32), classes=20):
    from paper_2311_11390_gb300 import alif, network
    alif.lib()
    w = synth.classification(seed=seed, B=B, T=T, dt=dt, hidden=hidden, classes=classes)
    net = network.ALIFNet.from_workload(w)
    words = torch.from_numpy(synth.pack_bits(w.S_in).view(np.int32)).cuda()
    labels = torch.from_numpy(w.labels.astype(np.int32)).cuda()
    keep = {}
    loss = net.loss(words, labels, T, keep=keep)
    for k in ("S0", "S1"):
        keep[k].retain_grad()
    loss.backward()
    torch.cuda.synchronize()
    assert alif.device_status() == 0
    return w, net, keep, loss


def _split_bound(W, S):
    """Per-output bound of the split-BF16 projection: sum_j |W_ij| S_j (2^-16 + (K+2) 2^-24)."""
    K = W.shape[1]
    return np.einsum("ij,bjt->bit", np.abs(W.astype(np.float64)), S.astype(np.float64)) * (
        2.0 ** -16 + (K + 2) * 2.0 ** -24) + 1e-6


@cuda
@pytest.mark.parametrize("seed, B, T, dt", [(0, 3, 300, 1.0), (1, 2, 700, 0.1)])
def test_network_forward_backward_matches_oracle(seed, B, T, dt):
    w, net, keep, loss = _run(seed, B, T, dt)
    S_in = w.S_in.astype(np.float64)
    nl = len(w.bias)
    S_prev = S_in
    forces = []
    for l in range(nl):
        I_gpu = keep[f"I{l}"].detach().cpu().numpy()
        I_o = oproj.project(w.W[l], S_prev, w.bias[l])
        assert np.all(np.abs(I_gpu - I_o) <= _split_bound(w.W[l], S_prev)), f"layer {l} projection"
        S_gpu = keep[f"S{l}"].detach().cpu().numpy()
        res = parity.compare_forward(S_gpu.astype(np.uint8), None, None, I_gpu, w.params[l], w.dt, w.arp)
        parity.assert_forward_parity(res)
        forces.append(res["force"])
        S_prev = S_gpu.astype(np.float64)
    # readout and loss from the GPU's last-layer spikes
    beta_o = onet.readout_beta(w.dt, w.tau_out)
    I_out = oproj.project(w.W[-1], S_prev, None)
    o = onet.readout_forward(I_out, beta_o)
    logits = keep["logits"].detach().cpu().numpy()
    np.testing.assert_allclose(logits, o, rtol=1e-5, atol=1e-5 * np.abs(o).max())
    L, g_o = onet.cross_entropy(o, w.labels)
    assert abs(float(loss.detach()) - L) <= 1e-5 * max(1.0, abs(L))
    # reverse chain in FP64 through the GPU's spikes
    g_Iout = onet.readout_backward(g_o, beta_o, w.S_in.shape[-1])
    gWo, gS, _ = oproj.project_backward(w.W[-1], S_prev, g_Iout)
    parity.grad_close(net.W_out.grad.cpu().numpy(), gWo, what="grad W_out")
    parity.grad_close(keep[f"S{nl - 1}"].grad.cpu().numpy(), gS, what=f"grad S{nl - 1}")
    for l in range(nl - 1, -1, -1):
        I_gpu = keep[f"I{l}"].detach().cpu().numpy()
        ob = ref.backward(I_gpu, parity.oracle_params(w.params[l]), w.dt, w.arp, gS, force=forces[l])
        for name, g in (("tau_mem", net.tau_mem[l].grad), ("tau_adapt", net.tau_adapt[l].grad),
                        ("theta0", net.theta0[l].grad), ("d", net.d[l].grad)):
            parity.grad_close(g.cpu().numpy(), getattr(ob, "g_" + name).sum(0), what=f"layer {l} {name}")
        S_below = S_in if l == 0 else keep[f"S{l - 1}"].detach().cpu().numpy().astype(np.float64)
        gW, gS_below, gb = oproj.project_backward(w.W[l], S_below, ob.gI)
        parity.grad_close(net.W[l].grad.cpu().numpy(), gW, what=f"layer {l} grad W")
        parity.grad_close(net.b[l].grad.cpu().numpy(), gb, what=f"layer {l} grad bias")
        if l > 0:
            parity.grad_close(keep[f"S{l - 1}"].grad.cpu().numpy(), gS_below, what=f"grad S{l - 1}")
        gS = gS_below


@cuda
def test_readout_and_loss_kernels_small():
    """The readout kernel against the oracle's step loop on a ragged T, and the loss kernel
    against the oracle's cross-entropy (including an out-of-range label giving NaN)."""
    from paper_2311_11390_gb300 import alif
    rng = np.random.default_rng(4)
    B, K, C, T = 3, 37, 5, 77
    S = rng.random((B, K, T)) < 0.1
    W = rng.standard_normal((C, K)).astype(np.float32)
    bias = rng.standard_normal(C).astype(np.float32)
    w_t, w_sum = alif.readout_weights(T, 1.0, 20.0, "cuda")
    words = torch.from_numpy(synth.pack_bits(S).view(np.int32)).cuda()
    Wt, bt = torch.from_numpy(W).cuda(), torch.from_numpy(bias).cuda()
    logits, counts = alif.readout_forward(words, T, Wt, bt, w_t, w_sum)
    beta = onet.readout_beta(1.0, 20.0)
    o = onet.readout_forward(oproj.project(W, S, bias), beta)
    np.testing.assert_allclose(logits.cpu().numpy(), o, rtol=1e-5, atol=1e-5 * np.abs(o).max())
    y = rng.integers(0, C, B)
    loss, g = alif.cross_entropy(logits, torch.from_numpy(y.astype(np.int32)).cuda())
    L, g_o = onet.cross_entropy(logits.cpu().numpy().astype(np.float64), y)
    assert abs(float(loss) - L) < 1e-5 * max(1.0, abs(L))
    np.testing.assert_allclose(g.cpu().numpy(), g_o, atol=1e-6)
    g_in = torch.from_numpy(g_o.astype(np.float32)).cuda()
    gS, gW, gb = alif.readout_backward(Wt, w_t, w_sum, counts, g_in, T)
    g_Io = onet.readout_backward(g_o, beta, T)
    gWo, gSo, gbo = oproj.project_backward(W, S, g_Io)
    np.testing.assert_allclose(gS.cpu().numpy(), gSo, rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(gW.cpu().numpy(), gWo, rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(gb.cpu().numpy(), gbo, rtol=1e-5, atol=1e-6)
    bad = torch.tensor([0, C, 1], dtype=torch.int32, device="cuda")
    lb, _ = alif.cross_entropy(logits, bad)
    assert torch.isnan(lb).all()
    packed = alif.pack_spikes(torch.from_numpy(S.astype(np.float32)).cuda())
    assert torch.equal(packed, words)
