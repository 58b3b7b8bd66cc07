"""Double-buffered host <-> device stepping gives every step the results of running it alone:
per-step inputs differ, so a slot reused too early (an upload over inputs still being read, a
compute over results still being downloaded) would show as a mismatch."""
import numpy as np
import pytest
import torch

from paper_2311_11390_gb300 import synth

pytestmark = pytest.mark.gpu
cuda = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")


@cuda
@pytest.mark.parametrize("n", [1, 2, 5])
def test_double_buffered_steps_match_serial(n):
    from paper_2311_11390_gb300 import alif
    from paper_2311_11390_gb300.pipeline import DoubleBuffered
    alif.lib()
    dev = torch.device("cuda")
    B, Nin, N, T = 2, 96, 160, 1500
    ws_ = [synth.feedforward(seed=s, B=B, Nin=Nin, N=N, T=T) for s in range(n)]
    w = ws_[0]
    table = alif.neuron_table(w.params.tau_mem, w.params.tau_adapt, w.params.theta0, w.params.d, w.params.R,
                              w.dt, w.arp, device=dev)
    Whi, Wlo = alif.split_bf16(torch.from_numpy(w.W).to(dev))
    bias = torch.from_numpy(w.bias).to(dev)
    gS = torch.from_numpy(np.random.default_rng(1).standard_normal((B, N, T), dtype=np.float32)).to(dev)
    hosts = [torch.from_numpy(synth.pack_bits(x.S_in).view(np.int32)).pin_memory() for x in ws_]
    I = torch.empty((B, N, T), device=dev)
    nw = (T + 31) // 32
    ckpt = torch.empty((B, N, alif.ckpt_count(T), 3), dtype=torch.int32, device=dev)
    ws = torch.empty(alif.workspace_size(B, N), dtype=torch.uint8, device=dev)
    gI = torch.empty_like(I)

    def run_step(S_dev, spikes, gp):
        alif.syn_project(S_dev, Whi, Wlo, bias, Nin=Nin, T=T, out=I)
        alif.forward_into(I, table, spikes, ckpt=ckpt)
        alif.backward(I, table, spikes, gS, ckpt=ckpt, workspace=ws, out_gI=gI, out_gp=gp)

    want = []
    for h in hosts:
        spikes = torch.empty((B, N, nw), dtype=torch.int32, device=dev)
        gp = torch.empty((5, N), device=dev)
        run_step(h.to(dev), spikes, gp)
        want.append((spikes.cpu(), gp.cpu()))

    got_s = [torch.empty((B, N, nw), dtype=torch.int32).pin_memory() for _ in range(n)]
    got_g = [torch.empty((5, N)).pin_memory() for _ in range(n)]
    pipe = DoubleBuffered(dev, lambda: {"S": torch.empty(hosts[0].shape, dtype=torch.int32, device=dev),
                                        "spikes": torch.empty((B, N, nw), dtype=torch.int32, device=dev),
                                        "gp": torch.empty((5, N), device=dev)})
    pipe.run(n,
             lambda k, sl: sl["S"].copy_(hosts[k], non_blocking=True),
             lambda k, sl: run_step(sl["S"], sl["spikes"], sl["gp"]),
             lambda k, sl: (got_s[k].copy_(sl["spikes"], non_blocking=True),
                            got_g[k].copy_(sl["gp"], non_blocking=True)))
    torch.cuda.synchronize()
    assert alif.device_status() == 0
    for k in range(n):
        assert torch.equal(got_s[k], want[k][0]), k
        assert torch.equal(got_g[k], want[k][1]), k
    if n > 1:
        assert not torch.equal(want[0][0], want[1][0])   # the steps' inputs differ
