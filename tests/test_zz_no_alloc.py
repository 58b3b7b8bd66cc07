"""The allocation-free backward entry point (alif_backward_noalloc).

It serves callers that cannot allocate device memory when they run the
backward pass; its scratch is a fixed array inside the library.  Collected
last on purpose.  It must give the same results as alif_backward() with a
caller workspace, call after call (the array keeps the previous call's
contents, which must not leak into the next result), and match the oracle's
FP64 BPTT at the gradient tolerances.

The host-side rejections at the end run without a GPU: every argument check
is made before the library makes any CUDA call, so the fake device pointers
they pass are never dereferenced.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import ref
from paper_2311_11390_gb300 import synth
from tests import parity

cuda = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")


def _setup(alif, seed, B, N, T):
    w = synth.population(seed=seed, B=B, N=N, T=T)
    table = alif.neuron_table(w.params.tau_mem, w.params.tau_adapt, w.params.theta0, w.params.d,
                              w.params.R, w.dt, w.arp)
    I = torch.from_numpy(w.I).cuda()
    return w, table, I, alif.forward(I, table)


def _noalloc(alif, I, table, out, gS, **kw):
    B, N, T = I.shape
    gI = torch.empty_like(I)
    ginit = torch.empty((B, N, 2), device="cuda")
    gp = torch.empty((5, N), device="cuda")
    alif.backward_noalloc(I, table, out["spikes"], gS, ckpt=out["ckpt"], out_gI=gI, out_ginit=ginit, out_gp=gp,
                          **kw)
    return gI, ginit, gp


@pytest.mark.gpu
@cuda
def test_noalloc_backward_matches_workspace_backward_and_oracle_twice():
    """Two calls in a row on different shapes: each equals alif_backward() with a workspace
    and the oracle's BPTT (dL/dI, parameter and initial-state gradients)."""
    from paper_2311_11390_gb300 import alif
    alif.lib()
    for seed, (B, N, T) in enumerate([(4, 64, 1000), (2, 96, 777)]):
        w, table, I, out = _setup(alif, seed, B, N, T)
        rng = np.random.default_rng(seed)
        gS_np = rng.standard_normal(I.shape).astype(np.float32)
        gS = torch.from_numpy(gS_np).cuda()
        gI_ref, ginit_ref, gp_ref = alif.backward(I, table, out["spikes"], gS, ckpt=out["ckpt"], want_ginit=True)
        gI, ginit, gp = _noalloc(alif, I, table, out, gS)
        torch.cuda.synchronize()
        assert alif.device_status() == 0
        torch.testing.assert_close(gI, gI_ref, rtol=1e-6, atol=1e-7)
        torch.testing.assert_close(ginit, ginit_ref, rtol=1e-6, atol=1e-7)
        torch.testing.assert_close(gp, gp_ref, rtol=1e-6, atol=1e-6)
        S = alif.unpack_spikes(out["spikes"], T).cpu().numpy()
        res = parity.compare_forward(S, None, None, w.I, w.params, w.dt, w.arp)
        parity.assert_forward_parity(res)
        ob = ref.backward(w.I, parity.oracle_params(w.params), w.dt, w.arp, gS_np.astype(np.float64),
                          force=res["force"])
        parity.grad_close(gI.cpu().numpy(), ob.gI, what="grad_I")
        for k, n in enumerate(["g_tau_mem", "g_tau_adapt", "g_theta0", "g_d", "g_R"]):
            parity.grad_close(gp[k].cpu().numpy(), getattr(ob, n).sum(0), what=n)
        p = np.exp(-w.dt / w.params.tau_adapt.astype(np.float64))
        parity.grad_close(ginit[..., 0].cpu().numpy(), ob.g_V0, what="grad_init_v")
        parity.grad_close(ginit[..., 1].cpu().numpy() * p[None, :], ob.g_a0, what="grad_init_a")


@pytest.mark.gpu
@cuda
def test_noalloc_trace_and_final_gradients():
    """grad_v, grad_a and grad_final reach the result as in alif_backward()."""
    from paper_2311_11390_gb300 import alif
    alif.lib()
    B, N, T = 2, 64, 1500
    w, table, I, out = _setup(alif, 7, B, N, T)
    g = torch.Generator(device="cuda").manual_seed(7)
    gS, gV, ga = (torch.randn(I.shape, device="cuda", generator=g) for _ in range(3))
    gf = torch.randn((B, N, 2), device="cuda", generator=g)
    gI_ref, ginit_ref, gp_ref = alif.backward(I, table, out["spikes"], gS, ckpt=out["ckpt"], grad_v=gV,
                                              grad_a=ga, grad_final=gf, want_ginit=True)
    gI, ginit, gp = _noalloc(alif, I, table, out, gS, grad_v=gV, grad_a=ga, grad_final=gf)
    torch.cuda.synchronize()
    assert alif.device_status() == 0
    torch.testing.assert_close(gI, gI_ref, rtol=1e-6, atol=1e-7)
    torch.testing.assert_close(ginit, ginit_ref, rtol=1e-6, atol=1e-7)
    torch.testing.assert_close(gp, gp_ref, rtol=1e-6, atol=1e-6)


@pytest.mark.gpu
@cuda
def test_noalloc_accepts_the_largest_batch_and_rejects_one_more_row():
    """B*N = 65536 (the array's capacity, every slot in use) matches alif_backward();
    65544 is refused with ALIF_ESHAPE before any work."""
    from paper_2311_11390_gb300 import alif
    alif.lib()
    B, N, T = 1024, 64, 96
    w, table, I, out = _setup(alif, 9, B, N, T)
    gS = torch.randn(I.shape, device="cuda", generator=torch.Generator(device="cuda").manual_seed(9))
    gI_ref, ginit_ref, gp_ref = alif.backward(I, table, out["spikes"], gS, ckpt=out["ckpt"], want_ginit=True)
    gI, ginit, gp = _noalloc(alif, I, table, out, gS)
    torch.cuda.synchronize()
    torch.testing.assert_close(gI, gI_ref, rtol=1e-6, atol=1e-7)
    torch.testing.assert_close(gp, gp_ref, rtol=1e-6, atol=1e-6)

    table8 = alif.neuron_table([20.0] * 8, [200.0] * 8, [1.0] * 8, [0.1] * 8, None, 0.1, 2.0)
    Ib = torch.zeros((65536 // 8 + 1, 8, 1), device="cuda")     # B*N = 65544
    spikes = torch.zeros((Ib.shape[0], 8, 1), dtype=torch.int32, device="cuda")
    with pytest.raises(alif.AlifError, match="ALIF_NOALLOC_MAX_ROWS"):
        alif.backward_noalloc(Ib, table8, spikes, torch.zeros_like(Ib))


@pytest.mark.gpu
@cuda
def test_noalloc_zero_steps_equals_workspace_backward():
    """T = 0: parameter gradients are zero and dL/d(init) = dL/d(final), as alif_backward()."""
    from paper_2311_11390_gb300 import alif
    alif.lib()
    B, N = 3, 16
    table = alif.neuron_table([20.0] * N, [200.0] * N, [1.0] * N, [0.1] * N, None, 0.1, 2.0)
    I = torch.zeros((B, N, 0), device="cuda")
    spikes = torch.zeros((B, N, 0), dtype=torch.int32, device="cuda")
    gf = torch.randn((B, N, 2), device="cuda")
    _, ginit_ref, gp_ref = alif.backward(I, table, spikes, I, grad_final=gf, want_gI=False, want_ginit=True)
    ginit = torch.full((B, N, 2), float("nan"), device="cuda")
    gp = torch.full((5, N), float("nan"), device="cuda")
    alif.backward_noalloc(I, table, spikes, I, grad_final=gf, out_ginit=ginit, out_gp=gp)
    torch.cuda.synchronize()
    assert torch.equal(ginit, ginit_ref) and torch.equal(ginit, gf)
    assert torch.equal(gp, gp_ref) and not gp.any()


def _call(L, B, N, T, I, slope=25.0):
    c = ctypes.c_void_p
    fake = c(1 << 20)  # 16-byte aligned; never dereferenced (every call below fails its checks first)
    return L.alif_backward_noalloc(B, N, T, I, fake, None, fake, fake, fake, None, None, None, slope, fake, None,
                                   fake, None)


def test_noalloc_host_side_rejections():
    """Refused on the host, before any CUDA call: a misaligned array (ALIF_ESHAPE), a
    non-finite or negative slope (ALIF_EINVAL), B*N over the limit, negative sizes."""
    from paper_2311_11390_gb300 import alif
    L = alif.lib()
    ok = ctypes.c_void_p(1 << 20)
    assert _call(L, 4, 64, 1000, ctypes.c_void_p((1 << 20) + 2)) == -3           # I misaligned
    assert _call(L, 4, 64, 1000, ok, slope=float("inf")) == -1
    assert _call(L, 4, 64, 1000, ok, slope=float("nan")) == -1
    assert _call(L, 4, 64, 1000, ok, slope=-1.0) == -1
    assert _call(L, 65536 // 8 + 1, 8, 10, ok) == -3
    assert _call(L, -1, 8, 10, ok) == -3
    assert _call(L, 1, 1 << 30, 1 << 20, ok) == -3                                 # also B*N*T > 2^40
    assert _call(L, 0, 64, 10, ok) == 0                                            # empty batch: nothing to do
