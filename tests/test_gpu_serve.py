"""Loss kernels of the fit requests, and the serving loop: continuous batching, admission by
device memory, and results that are the same alone and in a mix."""
import numpy as np
import pytest
import torch

from oracle import vanrossum as vr_oracle
from paper_2311_11390_gb300 import synth

pytestmark = pytest.mark.gpu
cuda = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")


def _alif():
    from paper_2311_11390_gb300 import alif
    alif.lib()
    return alif


@cuda
@pytest.mark.parametrize("T, chunk", [(1000, 256), (3001, 1024), (700, 4096)])
def test_vanrossum_kernels_match_oracle(T, chunk):
    alif = _alif()
    rng = np.random.default_rng(T)
    rows, dt, tau = 6, 0.1, 5.0
    x = rng.random((rows, T)) < 0.02
    y = rng.random((rows, T)) < 0.02
    xw = torch.from_numpy(synth.pack_bits(x).view(np.int32)).cuda()
    yw = torch.from_numpy(synth.pack_bits(y).view(np.int32)).cuda()
    nck = -(-T // chunk)
    fck = torch.empty((rows, nck), device="cuda")
    loss = torch.empty((rows,), device="cuda")
    alif.vanrossum_forward(xw, yw, T, dt, tau, chunk, fck, loss)
    ref_loss, ref_f = vr_oracle.forward(x, y, dt, tau)
    np.testing.assert_allclose(loss.cpu().numpy(), ref_loss, rtol=1e-5)
    g = np.zeros((rows, T), np.float32)
    gc = torch.zeros((rows,), device="cuda")
    for c in range(nck - 1, -1, -1):
        t0, t1 = c * chunk, min(T, (c + 1) * chunk)
        out = torch.empty((rows, t1 - t0), device="cuda")
        alif.vanrossum_backward(xw, yw, T, dt, tau, t0, t1, fck[:, c].contiguous(), gc, out)
        g[:, t0:t1] = out.cpu().numpy()
    ref_g = vr_oracle.backward(x, y, dt, tau)
    assert np.abs(g - ref_g).max() <= 1e-5 * max(1.0, np.abs(ref_g).max())


@cuda
def test_serving_same_alone_and_in_mix():
    """Continuous batching: each request's result is the same alone and in a mix (bitwise),
    although in the mix its rows share forward launches with other requests' rows."""
    from paper_2311_11390_gb300 import serve
    specs = serve.request_stream(10, seed=3, N_range=(64, 512), T_range=(1000, 6000), p_fit=0.4)
    reqs = [serve.make_request(rid, N, T, dt, fit, sd) for rid, N, T, dt, fit, sd, _ in specs]
    assert any(r.fit for r in reqs) and any(not r.fit for r in reqs)
    srv = serve.Server(max_active=4, chunk=1024, mem_budget=1 << 30, n_max=512)
    mixed, stats = srv.run(reqs, realtime=False)
    assert stats["requests"] == len(reqs) and stats["p99_s"] >= stats["p50_s"] > 0
    for r in reqs[:4]:
        alone, _ = serve.Server(max_active=1, chunk=1024, n_max=512).run([r], realtime=False)
        a, m = alone[r.rid], mixed[r.rid]
        assert np.array_equal(a.spikes, m.spikes)
        if r.fit:
            assert np.array_equal(a.loss, m.loss) and np.array_equal(a.grads, m.grads)
            assert np.isfinite(a.grads).all()
    assert alif_device_ok()


def alif_device_ok():
    alif = _alif()
    torch.cuda.synchronize()
    return alif.device_status() == 0


def _request_current(alif, r):
    """The request's FP32 current, computed alone by the library's projection (deterministic)."""
    from paper_2311_11390_gb300 import serve
    raster, W, bias, target = serve.materialize(r, torch.device("cuda"))
    hi, lo = alif.split_bf16(W)
    I = alif.syn_project(raster.unsqueeze(0), hi, lo, bias, Nin=serve.NIN, T=r.T)
    return I, target


@cuda
def test_serving_mix_matches_oracle():
    """A seeded mix of simulate and fit requests of different N, T and DT: every sampled
    request's spikes equal the FP64 oracle's on that request's current, and the fit requests'
    parameter gradients equal the oracle's BPTT driven by the oracle's van Rossum gradient."""
    alif = _alif()
    from oracle import ref
    from oracle import vanrossum as vr
    from paper_2311_11390_gb300 import serve
    from tests import parity
    specs = serve.request_stream(12, seed=9, N_range=(32, 160), T_range=(800, 3000), p_fit=0.5)
    reqs = [serve.make_request(rid, N, T, dt, fit, sd) for rid, N, T, dt, fit, sd, _ in specs]
    assert len({r.dt for r in reqs}) > 1 and any(r.fit for r in reqs)
    res, _ = serve.Server(max_active=5, chunk=512, mem_budget=1 << 30, n_max=256).run(reqs, realtime=False)
    for r in reqs:
        I, target = _request_current(alif, r)
        I_np = I.cpu().numpy()
        p = serve.request_params(r)
        S = synth.unpack_bits(res[r.rid].spikes[None], r.T)
        out = parity.compare_forward(S, None, None, I_np, p, r.dt, 2.0)
        parity.assert_forward_parity(out)
        if r.fit:
            Y = synth.unpack_bits(target.cpu().numpy().view(np.uint32)[None], r.T)[0]
            loss_o, _ = vr.forward(S[0], Y, r.dt, 5.0)
            np.testing.assert_allclose(res[r.rid].loss, loss_o, rtol=1e-5, atol=1e-7)
            gS = vr.backward(S[0], Y, r.dt, 5.0)[None]
            ob = ref.backward(I_np, parity.oracle_params(p), r.dt, 2.0, gS, force=out["force"], want_gI=False)
            for k, n in enumerate(["g_tau_mem", "g_tau_adapt", "g_theta0", "g_d", "g_R"]):
                parity.grad_close(res[r.rid].grads[k], getattr(ob, n)[0], what=f"request {r.rid} {n}")
    assert alif_device_ok()


@cuda
def test_serving_fit_gradient_matches_unchunked_backward():
    """A fit request's chunked pipeline (forward chunks, van Rossum, backward chunks last-first)
    gives the same parameter gradients as one unchunked forward/backward on the same current."""
    alif = _alif()
    from paper_2311_11390_gb300 import serve
    r = serve.make_request(0, 96, 3000, 0.1, True, seed=11)
    res, _ = serve.Server(max_active=1, chunk=1024, n_max=128).run([r], realtime=False)
    dev = torch.device("cuda")
    p = serve.request_params(r)
    table = alif.neuron_table(p.tau_mem, p.tau_adapt, p.theta0, p.d, p.R, r.dt, 2.0)
    I, tgt = _request_current(alif, r)
    out = alif.forward(I, table)
    assert np.array_equal(out["spikes"][0].cpu().numpy().view(np.uint32), res[0].spikes)
    fck = torch.empty((96, 1), device=dev)
    loss = torch.empty((96,), device=dev)
    alif.vanrossum_forward(out["spikes"][0], tgt, r.T, r.dt, 5.0, 4096, fck, loss)
    gS = torch.empty((96, r.T), device=dev)
    alif.vanrossum_backward(out["spikes"][0], tgt, r.T, r.dt, 5.0, 0, r.T, fck[:, 0].contiguous(),
                            torch.zeros(96, device=dev), gS)
    _, _, gp = alif.backward(I, table, out["spikes"], gS.unsqueeze(0), ckpt=out["ckpt"], want_gI=False)
    np.testing.assert_allclose(res[0].loss, loss.cpu().numpy(), rtol=1e-5)
    np.testing.assert_allclose(res[0].grads, gp.cpu().numpy(), rtol=1e-4, atol=1e-4 * np.abs(gp.cpu().numpy()).max())


@cuda
def test_serving_admission_respects_memory_budget():
    from paper_2311_11390_gb300 import serve
    reqs = [serve.make_request(k, 256, 2000, 0.1, False, seed=k) for k in range(6)]
    srv = serve.Server(max_active=6, chunk=1024, n_max=256)
    one = srv.footprint(reqs[0])
    srv.mem_budget = int(2.5 * one)          # at most two at a time
    seen = []
    res, stats = srv.run(reqs, realtime=False, on_done=lambda r: seen.append(r.rid))
    assert sorted(seen) == list(range(6))
    with pytest.raises(ValueError):
        serve.Server(mem_budget=one // 2, n_max=256).run([reqs[0]], realtime=False)
