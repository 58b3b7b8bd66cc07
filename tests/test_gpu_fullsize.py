"""Parity at the full sizes of the measured configurations, in the launch configuration the
bench times, on sampled rows the oracle computes one by one, plus properties checked on every
row.

* Feedforward layer (1000 Poisson inputs -> N=1024, B=32, T=16000, DT=0.1 ms, ARP=2 ms): split-BF16
  tcgen05 projection, block forward, block backward, exactly as the bench step calls them.  The
  oracle projects with its own split of the weights (hi = bf16(W), lo = bf16(W - hi)) in float64,
  so the GPU currents must match to FP32 accumulation rounding; forward and BPTT of the sampled rows
  run on the oracle's currents.  On every row: at most one spike in any T_eff consecutive steps.
* Neuron fit (1024 candidates, one OU current, T=400000, DT=0.05 ms, T_R=40): block forward and the
  parameter-only backward (grad_I = NULL) as the bench times them; sampled candidates' spikes and
  parameter gradients against the oracle.
"""
import numpy as np
import pytest
import torch

from oracle import project as oproj
from oracle import ref
from paper_2311_11390_gb300 import synth
from tests import parity

pytestmark = pytest.mark.gpu
cuda = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")


class _Sub:
    """Per-neuron parameters of the sampled rows (one oracle 'neuron' per sampled row)."""

    def __init__(self, p, idx):
        for k in ("tau_mem", "tau_adapt", "theta0", "d", "R"):
            v = getattr(p, k)
            setattr(self, k, None if v is None else np.asarray(v, np.float64)[idx])


def _min_isi_ok(S_words, T, teff):
    """At most one spike in any teff consecutive steps, on every row (bits unpacked on the host)."""
    bits = np.unpackbits(S_words.view(np.uint8), axis=-1, bitorder="little")[..., :T]
    rows, ts = np.nonzero(bits.reshape(-1, T))
    same = rows[1:] == rows[:-1]
    return bool(np.all(np.diff(ts)[same] >= teff)), int(bits.sum())


@cuda
def test_feedforward_full_size_sampled_rows():
    from paper_2311_11390_gb300 import alif
    alif.lib()
    B, Nin, N, T, dt, arp = 32, 1000, 1024, 16000, 0.1, 2.0
    w = synth.feedforward(seed=0, B=B, Nin=Nin, N=N, T=T, dt=dt, arp=arp)
    packed = synth.pack_bits(w.S_in)
    gS = np.random.default_rng(11).standard_normal((B, N, T), dtype=np.float32)
    dev = torch.device("cuda")
    table = alif.neuron_table(w.params.tau_mem, w.params.tau_adapt, w.params.theta0, w.params.d, w.params.R,
                              dt, arp, device=dev)
    S_dev = torch.from_numpy(packed.view(np.int32)).to(dev)
    W_dev = torch.from_numpy(w.W).to(dev)
    bias = torch.from_numpy(w.bias).to(dev)
    Whi, Wlo = alif.split_bf16(W_dev)
    I = torch.empty((B, N, T), device=dev)
    alif.syn_project(S_dev, Whi, Wlo, bias, Nin=Nin, T=T, out=I)
    out = alif.forward(I, table)
    gS_dev = torch.from_numpy(gS).to(dev)
    gI, _, _ = alif.backward(I, table, out["spikes"], gS_dev, ckpt=out["ckpt"])
    torch.cuda.synchronize()
    assert alif.device_status() == 0
    words = out["spikes"].cpu().numpy()
    ok, nspk = _min_isi_ok(words, T, max(alif.tr(dt, arp), 2))
    assert ok and nspk > 100000

    rng = np.random.default_rng(3)
    bs = rng.integers(0, B, 16)
    its = rng.choice(N, 16, replace=False)
    hi, lo = oproj.split_bf16(w.W[its])
    W_split = hi.astype(np.float64) + lo.astype(np.float64)
    I_o = np.stack([W_split[k] @ w.S_in[b].astype(np.float64) + float(w.bias[i])
                    for k, (b, i) in enumerate(zip(bs, its))])[None]            # [1, 16, T] float64
    I_g = I[torch.as_tensor(bs), torch.as_tensor(its)].cpu().numpy()[None]
    mag = np.stack([np.abs(W_split[k]) @ w.S_in[b].astype(np.float64) for k, b in enumerate(bs)])[None]
    lim = mag * (Nin + 2) * 2.0 ** -24 + 2.0 ** -23 * np.abs(I_o) + 1e-30
    assert np.all(np.abs(I_g - I_o) <= lim)
    I_o32 = I_o.astype(np.float32)
    S_g = np.unpackbits(words[bs, its].view(np.uint8), axis=-1, bitorder="little")[None, :, :T]
    P = _Sub(w.params, its)
    res = parity.compare_forward(S_g, None, None, I_o32, P, dt, arp)
    parity.assert_forward_parity(res)
    assert res["spikes"] > 100
    ob = ref.backward(I_o32, parity.oracle_params(P), dt, arp, gS[bs, its][None].astype(np.float64),
                      force=res["force"])
    parity.grad_close(gI[torch.as_tensor(bs), torch.as_tensor(its)].cpu().numpy()[None], ob.gI, what="grad_I")


@cuda
def test_neuron_fit_full_size_sampled_candidates():
    from paper_2311_11390_gb300 import alif
    alif.lib()
    N, T = 1024, 400000
    wf = synth.neuron_fit(seed=0, N=N, T=T)
    dev = torch.device("cuda")
    table = alif.neuron_table(wf.params.tau_mem, wf.params.tau_adapt, wf.params.theta0, wf.params.d, wf.params.R,
                              wf.dt, wf.arp, device=dev)
    I = torch.from_numpy(wf.I).to(dev)
    gS = np.random.default_rng(12).standard_normal((1, N, T), dtype=np.float32)
    spikes = torch.empty((1, N, (T + 31) // 32), dtype=torch.int32, device=dev)
    ckpt = torch.empty((1, N, alif.ckpt_count(T), 3), dtype=torch.int32, device=dev)
    gp = torch.empty((5, N), device=dev)
    alif.forward_into(I, table, spikes, ckpt=ckpt)
    alif.backward(I, table, spikes, torch.from_numpy(gS).to(dev), ckpt=ckpt, want_gI=False, out_gp=gp)
    torch.cuda.synchronize()
    assert alif.device_status() == 0
    words = spikes.cpu().numpy()
    ok, nspk = _min_isi_ok(words, T, max(alif.tr(wf.dt, wf.arp), 2))
    assert ok and nspk > 10000
    its = np.random.default_rng(4).choice(N, 4, replace=False)
    S_g = np.unpackbits(words[0, its].view(np.uint8), axis=-1, bitorder="little")[None, :, :T]
    I_rows = np.ascontiguousarray(wf.I[:, its])
    P = _Sub(wf.params, its)
    res = parity.compare_forward(S_g, None, None, I_rows, P, wf.dt, wf.arp)
    parity.assert_forward_parity(res)
    ob = ref.backward(I_rows, parity.oracle_params(P), wf.dt, wf.arp, gS[:, its].astype(np.float64),
                      force=res["force"], want_gI=False)
    g = gp.cpu().numpy()[:, its]
    for k, n in enumerate(["g_tau_mem", "g_tau_adapt", "g_theta0", "g_d", "g_R"]):
        parity.grad_close(g[k], getattr(ob, n)[0], what=n)
