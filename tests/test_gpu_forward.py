"""GPU parity of the block forward (and the plain sequential kernel) against the FP64 oracle.

All calls go through the C ABI (ctypes binding).  Inputs are the seeded
synthetic workloads; expected values come only from the oracle.
"""
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


def _run(alif, I, params, dt, arp, init=None, seq=False, want=True):
    table = alif.neuron_table(params.tau_mem, params.tau_adapt, params.theta0, params.d, params.R,
                              dt, arp)
    It = torch.from_numpy(np.ascontiguousarray(I)).cuda()
    out = alif.forward(It, table, init=init, want_v=want, want_a=want, seq=seq)
    torch.cuda.synchronize()
    assert alif.device_status() == 0
    T = I.shape[-1]
    S = alif.unpack_spikes(out["spikes"], T).cpu().numpy()
    V = out["v"].cpu().numpy() if want else None
    a = out["a"].cpu().numpy() if want else None
    return S, V, a, out


@cuda
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_population_config(seed):
    """B=8, N=128, T=1000, DT=0.1 ms, ARP=2 ms: bias U[0.8,1.6] + N(0, 0.3^2) noise."""
    alif = _alif()
    w = synth.population(seed=seed)
    S, V, a, out = _run(alif, w.I, w.params, w.dt, w.arp)
    res = parity.compare_forward(S, V, a, w.I, w.params, w.dt, w.arp)
    parity.assert_forward_parity(res)
    assert res["spikes"] > 1000
    # exactly one spike per nonzero bit and none past T
    assert S.shape == w.I.shape


@cuda
@pytest.mark.parametrize("T, arp, dt", [(1, 2.0, 0.1), (7, 0.3, 0.1), (255, 2.0, 0.1), (257, 1.0, 0.1),
                                        (1001, 2.0, 0.1), (1000, 0.1, 0.1), (2000, 0.2, 0.1),
                                        (3001, 40.0, 0.1), (777, 4.0, 0.05), (1024, 2.0, 1.0)])
def test_ragged_and_arp_edge_cases(T, arp, dt):
    """Ragged T (partial windows, T % 4 != 0 -> non-bulk path), T_R = 1, 2, 3, 20, 40, 80,
    400 (longer than a window), strong drive so that refractory spans cross windows."""
    alif = _alif()
    w = synth.population(seed=11, B=3, N=40, T=T, dt=dt, arp=arp, bias=(1.2, 3.0),
                         tau_mem=(2.0, 40.0), tau_adapt=(20.0, 400.0), d=(0.0, 0.8))
    S, V, a, _ = _run(alif, w.I, w.params, w.dt, w.arp)
    res = parity.compare_forward(S, V, a, w.I, w.params, w.dt, w.arp)
    parity.assert_forward_parity(res)


@cuda
def test_degenerate_time_constants_with_traces():
    """beta = 0, p = 0, subnormal decays, beta within 1e-6 of 1 (see the backward test of the same
    population): spikes, V and a traces against the oracle."""
    from tests.test_gpu_backward import _degenerate_population
    alif = _alif()
    w = _degenerate_population(seed=4, B=3, T=1100)
    S, V, a, _ = _run(alif, w.I, w.params, w.dt, w.arp)
    assert np.isfinite(V).all() and np.isfinite(a).all()
    res = parity.compare_forward(S, V, a, w.I, w.params, w.dt, w.arp)
    parity.assert_forward_parity(res)
    assert res["spikes"] > 1000


@cuda
def test_nonrest_initial_state():
    alif = _alif()
    w = synth.population(seed=5, B=2, N=64, T=900)
    rng = np.random.default_rng(0)
    S0 = rng.random((2, 64)) < 0.3
    V0 = rng.uniform(-0.5, 1.0, (2, 64))
    teff = max(alif.tr(w.dt, w.arp), 2)
    v = np.where(S0, 0.0, V0).astype(np.float32)
    a = S0.astype(np.float32)
    rem = np.where(S0, teff - 1, 0)
    init = alif.state_tensor(2, 64, v=torch.from_numpy(v), a=torch.from_numpy(a), rem=torch.from_numpy(rem))
    S, V, A, _ = _run(alif, w.I, w.params, w.dt, w.arp, init=init)
    oinit = parity.oracle_init_from_state(v, a, rem, teff)
    res = parity.compare_forward(S, V, A, w.I, w.params, w.dt, w.arp, init=oinit)
    parity.assert_forward_parity(res)


@cuda
def test_feedforward_currents_config_subset():
    """Currents of the feedforward workload (Poisson inputs through N(0, 2/1000) weights plus
    bias), computed by the FP64 projection oracle and rounded to FP32; T_R = 10, 20, 40."""
    alif = _alif()
    for arp in (1.0, 2.0, 4.0):
        w = synth.feedforward(seed=3, B=4, N=96, T=4000, arp=arp)
        I = project.project(w.W, w.S_in, w.bias).astype(np.float32)
        S, V, a, _ = _run(alif, I, w.params, w.dt, w.arp)
        res = parity.compare_forward(S, V, a, I, w.params, w.dt, w.arp)
        parity.assert_forward_parity(res)
        assert res["spikes"] > 100


@cuda
def test_neuron_fit_config_subset():
    """OU-driven candidates at DT=0.05 ms, T_R=40, heterogeneous theta0, d, R (shortened T)."""
    alif = _alif()
    w = synth.neuron_fit(seed=0, N=64, T=40000)
    S, V, a, _ = _run(alif, w.I, w.params, w.dt, w.arp)
    res = parity.compare_forward(S, V, a, w.I, w.params, w.dt, w.arp)
    parity.assert_forward_parity(res)
    assert res["spikes"] > 200


@cuda
def test_chunked_equals_single_run():
    """Forward over [0, T1) then [T1, T) from the returned state equals one run over [0, T)."""
    alif = _alif()
    w = synth.population(seed=9, B=2, N=64, T=2048)
    table = alif.neuron_table(w.params.tau_mem, w.params.tau_adapt, w.params.theta0, w.params.d,
                              w.params.R, w.dt, w.arp)
    It = torch.from_numpy(w.I).cuda()
    full = alif.forward(It, table, want_v=True)
    T1 = 768
    a = alif.forward(It[..., :T1].contiguous(), table, want_v=True)
    b = alif.forward(It[..., T1:].contiguous(), table, init=a["final"], want_v=True)
    S_full = alif.unpack_spikes(full["spikes"], 2048)
    S_ab = torch.cat([alif.unpack_spikes(a["spikes"], T1), alif.unpack_spikes(b["spikes"], 2048 - T1)], -1)
    assert torch.equal(S_full, S_ab)
    torch.testing.assert_close(torch.cat([a["v"], b["v"]], -1), full["v"], rtol=1e-6, atol=1e-6)
    # checkpoints of the single run equal the chunk states at window boundaries
    ck = full["ckpt"]
    assert torch.equal(ck[:, :, T1 // 256], a["final"])


@cuda
@pytest.mark.parametrize("seed, seq", [(0, True), (1, True), (0, "staged"), (1, "staged")])
def test_sequential_comparator(seed, seq):
    """The plain per-step kernel (and its staged variant) is the same model in
    uncompensated FP32 (no exact re-decision, a carried step by step): spikes agree
    with the oracle except at crossings within 1e-4 of threshold, traces within 1e-4."""
    alif = _alif()
    w = synth.population(seed=seed)
    S, V, a, _ = _run(alif, w.I, w.params, w.dt, w.arp, seq=seq)
    res = parity.compare_forward(S, V, a, w.I, w.params, w.dt, w.arp, flip_margin=1e-4,
                                 trace_rtol=1e-4)
    assert not res["bad"], res["bad"][:3]


@cuda
@pytest.mark.parametrize("B, N, T", [(1, 33, 31), (3, 50, 97), (2, 64, 1000)])
def test_staged_sequential_matches_plain(B, N, T):
    """Ragged row groups (rows not a multiple of 32) and ragged 32-step tiles: the staged
    kernel runs the plain kernel's arithmetic in the same order, so spikes, traces and the
    final state are bit-identical to it."""
    alif = _alif()
    w = synth.population(seed=5, B=B, N=N, T=T)
    table = alif.neuron_table(w.params.tau_mem, w.params.tau_adapt, w.params.theta0, w.params.d,
                              w.params.R, w.dt, w.arp)
    It = torch.from_numpy(w.I).cuda()
    o1 = alif.forward(It, table, want_v=True, want_a=True, seq=True)
    o2 = alif.forward(It, table, want_v=True, want_a=True, seq="staged")
    for k in ("spikes", "v", "a", "final"):
        assert torch.equal(o1[k], o2[k]), k


@cuda
def test_empty_and_degenerate_shapes():
    alif = _alif()
    w = synth.population(seed=1, B=2, N=8, T=10)
    table = alif.neuron_table(w.params.tau_mem, w.params.tau_adapt, w.params.theta0, w.params.d,
                              w.params.R, w.dt, w.arp)
    empty = torch.empty((2, 8, 0), dtype=torch.float32, device="cuda")
    out = alif.forward(empty, table)
    assert out["spikes"].shape == (2, 8, 0)
    v, a, rem = alif.state_fields(out["final"])
    assert torch.all(v == 0) and torch.all(a == 0) and torch.all(rem == 0)
    zero_b = torch.empty((0, 8, 10), dtype=torch.float32, device="cuda")
    alif.forward(zero_b, table)
    with pytest.raises(alif.AlifError):
        alif.neuron_table(w.params.tau_mem, w.params.tau_adapt, -w.params.theta0, w.params.d,
                          w.params.R, w.dt, w.arp)
    with pytest.raises(alif.AlifError):
        alif.tr(0.3, 1.0)


@cuda
@pytest.mark.parametrize("T, arp, dt, seed", [(16, 2.0, 0.1, 5), (512, 1.0, 0.1, 3), (528, 4.0, 1.0, 6),
                                              (1024, 2.0, 0.1, 0), (2000, 0.2, 0.1, 1), (3008, 40.0, 0.1, 2),
                                              (4096, 2.0, 0.05, 4)])
def test_window_lengths_agree(T, arp, dt, seed):
    """The 512-step kernel (chosen for few rows; calls without traces) and the 256-step kernel:
    both give the oracle's spikes, and the same checkpoints (refractory counts exactly, v and a
    within FP32 rounding of the two scans) and final states; the 512-step kernel records the
    middle checkpoint of each window from the round that covers it."""
    alif = _alif()
    w = synth.population(seed=seed, B=3, N=40, T=T, dt=dt, arp=arp, bias=(1.2, 3.0),
                         tau_mem=(2.0, 40.0), tau_adapt=(20.0, 400.0), d=(0.0, 0.8))
    outs = {}
    for win in (256, 512):
        prev = alif.forward_window(win)
        try:
            S, _, _, out = _run(alif, w.I, w.params, w.dt, w.arp, want=False)
        finally:
            alif.forward_window(prev)
        res = parity.compare_forward(S, None, None, w.I, w.params, w.dt, w.arp)
        parity.assert_forward_parity(res)
        outs[win] = (S, out["ckpt"].cpu().numpy(), out["final"].cpu().numpy())
    (S8, c8, f8), (S16, c16, f16) = outs[256], outs[512]
    assert np.array_equal(S8, S16)
    for a, b in ((c8, c16), (f8, f16)):
        assert np.array_equal(a[..., 2], b[..., 2])
        av = np.ascontiguousarray(a).view(np.float32)[..., :2]
        bv = np.ascontiguousarray(b).view(np.float32)[..., :2]
        assert np.allclose(av, bv, rtol=1e-5, atol=1e-6)


@cuda
def test_wide_windows_initial_state_and_chunks():
    """The 512-step kernel from a non-rest initial state (spikes against the oracle), and two chunked
    calls (the second from the first's final state, chunk boundary in the middle of a window) against
    one call: spikes equal, states within FP32 rounding of the two window partitions."""
    alif = _alif()
    prev = alif.forward_window(512)
    try:
        w = synth.population(seed=5, B=2, N=64, T=1024)
        rng = np.random.default_rng(1)
        S0 = rng.random((2, 64)) < 0.3
        V0 = rng.uniform(-0.5, 1.0, (2, 64))
        teff = max(alif.tr(w.dt, w.arp), 2)
        v = np.where(S0, 0.0, V0).astype(np.float32)
        a = S0.astype(np.float32)
        rem = np.where(S0, teff - 1, 0)
        init = alif.state_tensor(2, 64, v=torch.from_numpy(v), a=torch.from_numpy(a), rem=torch.from_numpy(rem))
        S, _, _, _ = _run(alif, w.I, w.params, w.dt, w.arp, init=init, want=False)
        res = parity.compare_forward(S, None, None, w.I, w.params, w.dt, w.arp,
                                     init=parity.oracle_init_from_state(v, a, rem, teff))
        parity.assert_forward_parity(res)

        w = synth.population(seed=9, B=2, N=64, T=2048)
        table = alif.neuron_table(w.params.tau_mem, w.params.tau_adapt, w.params.theta0, w.params.d,
                                  w.params.R, w.dt, w.arp)
        It = torch.from_numpy(w.I).cuda()
        full = alif.forward(It, table)
        T1 = 768
        c1 = alif.forward(It[..., :T1].contiguous(), table)
        c2 = alif.forward(It[..., T1:].contiguous(), table, init=c1["final"])
        S_full = alif.unpack_spikes(full["spikes"], 2048)
        S_ab = torch.cat([alif.unpack_spikes(c1["spikes"], T1), alif.unpack_spikes(c2["spikes"], 2048 - T1)], -1)
        assert torch.equal(S_full, S_ab)
        ck = np.ascontiguousarray(full["ckpt"][:, :, T1 // 256].cpu().numpy())
        fin = np.ascontiguousarray(c1["final"].cpu().numpy())
        assert np.array_equal(ck[..., 2], fin[..., 2])
        assert np.allclose(ck.view(np.float32)[..., :2], fin.view(np.float32)[..., :2], rtol=1e-5, atol=1e-6)
        assert np.array_equal(full["final"].cpu().numpy()[..., 2], c2["final"].cpu().numpy()[..., 2])
    finally:
        alif.forward_window(prev)
