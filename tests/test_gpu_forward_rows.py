"""GPU parity of the lane-per-row block forward (K-step Blocks inside a lane) against the FP64
oracle, and its agreement with the warp-per-row kernel.

All calls go through the C ABI (ctypes binding) with the layout forced; inputs are the seeded
synthetic workloads, expected spikes come only from the oracle.
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


def _run(alif, layout, I, table, init=None):
    prev = alif.forward_layout(layout)
    try:
        It = torch.from_numpy(np.ascontiguousarray(I)).cuda()
        alif.forward_stats()  # clear the counters
        out = alif.forward(It, table, init=init)
        torch.cuda.synchronize()
        stats = alif.forward_stats()
    finally:
        alif.forward_layout(prev)
    assert alif.device_status() == 0
    S = alif.unpack_spikes(out["spikes"], I.shape[-1]).cpu().numpy()
    return S, out, stats


def _table(alif, w):
    return alif.neuron_table(w.params.tau_mem, w.params.tau_adapt, w.params.theta0, w.params.d, w.params.R,
                             w.dt, w.arp)


def _states_close(a, b):
    a = np.ascontiguousarray(a.cpu().numpy())
    b = np.ascontiguousarray(b.cpu().numpy())
    assert np.array_equal(a[..., 2], b[..., 2])
    assert np.allclose(a.view(np.float32)[..., :2], b.view(np.float32)[..., :2], rtol=1e-5, atol=1e-6)


@cuda
@pytest.mark.parametrize("T, arp, dt, seed", [(4, 2.0, 0.1, 0), (60, 2.0, 0.1, 1), (64, 0.1, 0.1, 2),
                                              (100, 0.2, 0.1, 3), (256, 0.3, 0.1, 4), (1000, 0.4, 0.1, 5),
                                              (1028, 0.5, 0.1, 6), (1000, 0.7, 0.1, 7), (2000, 0.8, 0.1, 8),
                                              (3008, 2.0, 0.1, 9), (4096, 4.0, 0.1, 10), (1024, 40.0, 0.1, 11),
                                              (528, 4.0, 1.0, 12), (4096, 2.0, 0.05, 13), (2000, 1.0, 0.1, 14),
                                              (1004, 1.5, 0.1, 15), (1600, 1.6, 0.1, 16)])
def test_lane_layout_matches_oracle_and_warp_layout(T, arp, dt, seed):
    """T_R = 1 .. 400 (Blocks of K = 16, 8, 4 and 2 steps by T_eff, including T_eff = K), T a multiple of
    4 with partial last Blocks and stages, rows not a multiple of 32 (idle lanes), strong drive
    and slow membranes so that refractory spans cross Blocks and stages: the oracle's spikes, and
    checkpoints and final states equal to the warp-per-row kernel's (refractory counts exactly,
    v and a within FP32 rounding)."""
    alif = _alif()
    w = synth.population(seed=seed, B=3, N=40, T=T, dt=dt, arp=arp, bias=(1.2, 3.0),
                         tau_mem=(2.0, 40.0), tau_adapt=(20.0, 400.0), d=(0.0, 0.8))
    table = _table(alif, w)
    S2, o2, st2 = _run(alif, 2, w.I, table)
    res = parity.compare_forward(S2, None, None, w.I, w.params, w.dt, w.arp)
    parity.assert_forward_parity(res)
    assert st2["rows"] == 3 * 40
    S1, o1, _ = _run(alif, 1, w.I, table)
    assert np.array_equal(S1, S2)
    _states_close(o1["ckpt"], o2["ckpt"])
    _states_close(o1["final"], o2["final"])


@cuda
@pytest.mark.parametrize("seed", [0, 1])
def test_lane_layout_population_config(seed):
    """B=8, N=128, T=1000, DT=0.1 ms, ARP=2 ms (1024 rows, 32 warps) through the lane kernel."""
    alif = _alif()
    w = synth.population(seed=seed)
    S, out, stats = _run(alif, 2, w.I, _table(alif, w))
    res = parity.compare_forward(S, None, None, w.I, w.params, w.dt, w.arp)
    parity.assert_forward_parity(res)
    assert res["spikes"] > 1000
    assert stats["rows"] == 8 * 128


@cuda
def test_lane_layout_feedforward_workload():
    """Currents of the feedforward workload (Poisson inputs through N(0, 2/1000) weights plus bias,
    from the FP64 projection oracle rounded to FP32) at N=1024, T=4096: oracle spikes; the
    re-decided margins are counted."""
    alif = _alif()
    w = synth.feedforward(seed=3, B=1, Nin=1000, N=1024, T=4096, dt=0.1, arp=2.0)
    I = project.project(w.W, w.S_in, w.bias).astype(np.float32)
    S, out, stats = _run(alif, 2, I, _table(alif, w))
    res = parity.compare_forward(S, None, None, I, w.params, w.dt, w.arp)
    parity.assert_forward_parity(res)
    assert res["spikes"] > 3000
    assert stats["exact_spikes"] <= stats["exact_checks"]


@cuda
def test_lane_layout_initial_state_and_chunks():
    """From a non-rest initial state (refractory counts > 0 at the start) against the oracle, and two
    chunked calls (the second from the first's final state, the boundary inside a stage and inside a
    Block of 8) against one call: spikes equal, states within FP32 rounding."""
    alif = _alif()
    w = synth.population(seed=5, B=2, N=64, T=1024)
    rng = np.random.default_rng(1)
    S0 = rng.random((2, 64)) < 0.3
    V0 = rng.uniform(-0.5, 1.0, (2, 64))
    teff = max(alif.tr(w.dt, w.arp), 2)
    v = np.where(S0, 0.0, V0).astype(np.float32)
    a = S0.astype(np.float32)
    rem = np.where(S0, teff - 1, 0)
    init = alif.state_tensor(2, 64, v=torch.from_numpy(v), a=torch.from_numpy(a), rem=torch.from_numpy(rem))
    table = _table(alif, w)
    S, _, _ = _run(alif, 2, w.I, table, init=init)
    res = parity.compare_forward(S, None, None, w.I, w.params, w.dt, w.arp,
                                 init=parity.oracle_init_from_state(v, a, rem, teff))
    parity.assert_forward_parity(res)

    w = synth.population(seed=9, B=2, N=64, T=2048)
    table = _table(alif, w)
    _, full, _ = _run(alif, 2, w.I, table)
    T1 = 772  # a multiple of 4, not of 8 or 64
    _, c1, _ = _run(alif, 2, w.I[..., :T1], table)
    _, c2, _ = _run(alif, 2, w.I[..., T1:], table, init=c1["final"])
    S_full = alif.unpack_spikes(full["spikes"], 2048)
    S_ab = torch.cat([alif.unpack_spikes(c1["spikes"], T1), alif.unpack_spikes(c2["spikes"], 2048 - T1)], -1)
    assert torch.equal(S_full, S_ab)
    _states_close(full["final"], c2["final"])


@cuda
def test_lane_layout_declines_unstageable_calls():
    """T % 4 != 0 cannot be staged by TMA: with the lane layout forced the call is served by the
    warp-per-row kernel (still the oracle's spikes)."""
    alif = _alif()
    w = synth.population(seed=4, B=2, N=48, T=1001)
    S, _, _ = _run(alif, 2, w.I, _table(alif, w))
    res = parity.compare_forward(S, None, None, w.I, w.params, w.dt, w.arp)
    parity.assert_forward_parity(res)


@cuda
@pytest.mark.parametrize("arp", [0.3, 2.0])
def test_lane_layout_fast_membranes(arp):
    """tau_mem of 0.005 - 0.02 ms at DT = 0.1 ms (beta^K below 2^-100): refractory lanes recompute the
    masked input chain instead of entering with the effective membrane; the oracle's spikes."""
    alif = _alif()
    w = synth.population(seed=21, B=2, N=48, T=2000, dt=0.1, arp=arp, tau_mem=(0.005, 0.02), bias=(0.9, 2.0))
    S, _, stats = _run(alif, 2, w.I, _table(alif, w))
    res = parity.compare_forward(S, None, None, w.I, w.params, w.dt, w.arp)
    parity.assert_forward_parity(res)
    assert res["spikes"] > 1000
    assert stats["rows"] == 2 * 48
