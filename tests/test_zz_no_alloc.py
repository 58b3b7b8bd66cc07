"""The allocation-free backward entry point (alif_backward_noalloc).

It serves callers that cannot allocate device memory when they run the
backward pass; its scratch is a fixed array inside the library.  Collected
last on purpose.  It must give the same results as alif_backward() with a
caller workspace, call after call (the array keeps the previous call's
contents, which must not leak into the next result).
"""
import numpy as np
import pytest
import torch

from paper_2311_11390_gb300 import synth

cuda = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")


@pytest.mark.gpu
@cuda
def test_noalloc_backward_matches_workspace_backward_twice():
    from paper_2311_11390_gb300 import alif
    alif.lib()
    for seed, (B, N, T) in enumerate([(4, 64, 1000), (2, 96, 777)]):
        w = synth.population(seed=seed, B=B, N=N, T=T)
        table = alif.neuron_table(w.params.tau_mem, w.params.tau_adapt, w.params.theta0, w.params.d,
                                  w.params.R, w.dt, w.arp)
        I = torch.from_numpy(w.I).cuda()
        out = alif.forward(I, table)
        g = torch.Generator(device="cuda").manual_seed(seed)
        gS = torch.randn(I.shape, device="cuda", generator=g)
        gI_ref, ginit_ref, gp_ref = alif.backward(I, table, out["spikes"], gS, ckpt=out["ckpt"], want_ginit=True)
        gI = torch.empty_like(I)
        ginit = torch.empty((B, N, 2), device="cuda")
        gp = torch.empty((5, N), device="cuda")
        alif.backward_noalloc(I, table, out["spikes"], gS, ckpt=out["ckpt"], out_gI=gI, out_ginit=ginit, out_gp=gp)
        torch.cuda.synchronize()
        assert alif.device_status() == 0
        torch.testing.assert_close(gI, gI_ref, rtol=1e-6, atol=1e-7)
        torch.testing.assert_close(ginit, ginit_ref, rtol=1e-6, atol=1e-7)
        torch.testing.assert_close(gp, gp_ref, rtol=1e-6, atol=1e-6)


@pytest.mark.gpu
@cuda
def test_noalloc_rejects_batches_over_the_limit():
    from paper_2311_11390_gb300 import alif
    alif.lib()
    table = alif.neuron_table([20.0] * 8, [200.0] * 8, [1.0] * 8, [0.1] * 8, None, 0.1, 2.0)
    I = torch.zeros((65536 // 8 + 1, 8, 1), device="cuda")     # B*N = 65544 > 65536
    z = torch.zeros_like(I)
    spikes = torch.zeros((I.shape[0], 8, 1), dtype=torch.int32, device="cuda")
    with pytest.raises(alif.AlifError, match="ALIF_NOALLOC_MAX_ROWS"):
        alif.backward_noalloc(I, table, spikes, z)
