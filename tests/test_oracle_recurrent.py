"""Pins of the oracle's recurrent layer (Section 2, Eq 3's recurrent term with transmission
latency D = T_R; Prop 3's recurrent current between Blocks).

Independent of the oracle's code: the reduction to the feedforward layer when W_rec = 0, a
closed form for one presynaptic spike arriving T_R steps later, and the paper's blocked form
(Props 1-5 with Prop 3's recurrent current from the previous Block's spikes) written out
separately over a whole population.
"""
import math

import numpy as np
import pytest

from paper_2311_11390_gb300 import synth


def _params(N, tau_mem, tau_adapt, theta0, d, R=1.0):
    from oracle.ref import Params
    f = lambda v: np.full(N, v, np.float64) if np.isscalar(v) else np.asarray(v, np.float64)
    return Params(f(tau_mem), f(tau_adapt), f(theta0), f(d), f(R))


def _w_rec(rng, N, scale):
    return (scale * rng.standard_normal((N, N)) / math.sqrt(N)).astype(np.float32)


@pytest.mark.parametrize("arp", [2.0, 0.1])
def test_recurrent_without_weights_is_feedforward(oracle_lib, arp):
    """W_rec = 0: the recurrent layer is the feedforward layer, bit for bit."""
    ref = oracle_lib
    w = synth.population(seed=5, B=2, N=16, T=700, arp=arp, tau_adapt=(60.0, 300.0), d=(0.0, 0.5))
    P = ref.Params(*w.params.astype32().__dict__.values())
    ff = ref.forward(w.I, P, w.dt, w.arp)
    rec = ref.forward_recurrent(w.I, np.zeros((16, 16), np.float32), P, w.dt, w.arp)
    assert ff.S.sum() > 20
    assert np.array_equal(ff.S, rec.S)
    assert np.array_equal(ff.V, rec.V) and np.array_equal(ff.a, rec.a)
    assert np.array_equal(rec.I_total, w.I.astype(np.float64))


@pytest.mark.parametrize("arp, dt", [(2.0, 0.1), (1.0, 0.5), (0.1, 0.1)])
def test_one_presynaptic_spike_arrives_T_R_later(oracle_lib, arp, dt):
    """Neuron 0 (d = 0, constant drive from rest) first fires at k* = floor(t*/DT) + 1 (LIF
    closed form); neuron 1 has no feedforward input and one synapse w from neuron 0.  Its
    current is w exactly from step k* + T_R on (Section 2: D = T_R), so V_1 is 0 before and
    (1 - beta) R w at that step (Eq 2)."""
    ref = oracle_lib
    TR = ref.tr(dt, arp)
    tau, th0, R, I0, w = 20.0, 1.0, 1.3, 1.7, 0.25
    I32 = np.float32(I0)
    tstar = -tau * math.log(1.0 - th0 / (R * float(I32)))
    assert abs(tstar / dt - round(tstar / dt)) > 1e-6
    kstar = math.floor(tstar / dt) + 1          # paper time of neuron 0's first spike
    T = kstar + TR + 5
    I = np.zeros((1, 2, T), np.float32)
    I[0, 0] = I32
    W = np.zeros((2, 2), np.float32)
    W[1, 0] = np.float32(w)
    out = ref.forward_recurrent(I, W, _params(2, tau, 500.0, th0, 0.0, R), dt, arp)
    assert int(np.flatnonzero(out.S[0, 0])[0]) + 1 == kstar
    k_arrive = kstar + TR                        # paper time of the first recurrent input
    assert np.all(out.V[0, 1, :k_arrive - 1] == 0.0)
    beta = math.exp(-dt / tau)
    assert out.V[0, 1, k_arrive - 1] == pytest.approx((1 - beta) * R * float(np.float32(w)), rel=1e-14)
    assert out.I_total[0, 1, k_arrive - 1] == float(np.float32(w))
    assert np.all(out.I_total[0, 1, :k_arrive - 1] == 0.0)


def _blocks_recurrent(I_ff, W, beta, p, th0, d, R, TR):
    """Section 3 over a population with recurrent synapses.  Block n+1's input current is
    Prop 3's: bias and feedforward current plus W_rec times the spikes of Block n at the same
    in-Block step, gated by the ARP mask 1{z_n >= max S_n}.  Inside a Block the no-reset
    membrane is Prop 1's convolution, the first spike comes from phi (Prop 2, Eq 9), and the
    membrane and adaptation carries are Props 4 and 5.  I_ff zero-padded to a multiple of T_R."""
    N, T = I_ff.shape
    nb = -(-T // TR)
    x = np.zeros((N, nb * TR))
    x[:, :T] = np.asarray(I_ff, np.float64)
    t = np.arange(1, TR + 1)
    K = np.tril(beta[:, None, None] ** (t[None, :, None] - t[None, None, :]))   # [N, TR, TR]
    K = np.where(np.tril(np.ones((TR, TR), bool))[None], K, 0.0)
    W64 = np.asarray(W, np.float64)
    S_all = np.zeros((N, nb * TR), np.int64)
    V0, a0 = np.zeros(N), np.zeros(N)
    z_prev, S_prev = np.zeros((N, TR)), np.zeros((N, TR))
    for n in range(nb):
        cur = x[:, n * TR:(n + 1) * TR] + W64 @ S_prev                   # Prop 3 currents
        mask = (z_prev >= S_prev.max(axis=1, keepdims=True)).astype(np.float64)
        drive = (R[:, None] * cur) * mask
        Vt = beta[:, None] ** t[None] * V0[:, None] + (1 - beta[:, None]) * np.einsum("ntj,nj->nt", K, drive)
        theta = th0[:, None] + d[:, None] * p[:, None] ** t[None] * a0[:, None]
        St = (Vt > theta).astype(np.int64)
        z = np.cumsum(np.cumsum(St, axis=1), axis=1)                     # Prop 2
        S = (z == 1).astype(np.int64)
        for i in range(N):
            if S[i].any():
                ts = int(np.argmax(S[i])) + 1
                a_s = p[i] ** ts * a0[i]
                a0[i] = p[i] ** (TR - ts) * (a_s + 1.0 / p[i])           # Prop 5, spiked
                V0[i] = 0.0                                              # Prop 4, spiked
            else:
                a0[i] = p[i] ** TR * a0[i]
                V0[i] = Vt[i, -1]
        S_all[:, n * TR:(n + 1) * TR] = S
        z_prev, S_prev = z.astype(np.float64), S.astype(np.float64)
    return S_all[:, :T]


@pytest.mark.parametrize("seed, arp, scale", [(0, 2.0, 1.5), (1, 1.0, 3.0), (2, 4.0, 2.0), (3, 0.3, -2.0)])
def test_recurrent_oracle_equals_paper_blocks(oracle_lib, seed, arp, scale):
    """Props 1-5 with Prop 3's recurrent current reproduce the oracle's spike trains exactly
    (no FP64 near-ties in these cases, asserted), excitatory and inhibitory coupling."""
    ref = oracle_lib
    N = 24
    w = synth.population(seed=seed, B=2, N=N, T=801, arp=arp, bias=(1.1, 2.2), tau_adapt=(60.0, 300.0),
                         d=(0.0, 0.6))
    Wr = _w_rec(np.random.default_rng(seed + 100), N, scale)
    P = ref.Params(*w.params.astype32().__dict__.values())
    out = ref.forward_recurrent(w.I, Wr, P, w.dt, w.arp)
    ff = ref.forward(w.I, P, w.dt, w.arp)
    TR = ref.tr(w.dt, w.arp)
    assert out.S.sum() > 50
    assert not np.array_equal(out.S, ff.S)          # the coupling changes the trains
    assert np.abs(out.margin).min() > 1e-9
    tm, ta, th0, d, R = (np.asarray(v, np.float64) for v in P.arrays())
    beta, p = np.exp(-w.dt / tm), np.exp(-w.dt / ta)
    for b in range(2):
        S = _blocks_recurrent(w.I[b], Wr, beta, p, th0, d, R, TR)
        assert np.array_equal(S, out.S[b]), b


def test_recurrent_strict_threshold_at_exact_tie(oracle_lib):
    """Eq 1 is strict in the recurrent layer too.  Neuron 1 has no feedforward input, d = 0 and
    one synapse w from neuron 0; at the step the first recurrent input arrives its membrane is
    ((1 - beta) R) w evaluated in binary64 with beta = exp(-DT/tau) (the oracle's operations,
    in that order), and its threshold theta0 is set to exactly that value: V = theta, no spike."""
    ref = oracle_lib
    dt, arp, tau, R, I0, w = 0.1, 2.0, 20.0, 1.3, 1.7, 0.25
    TR = ref.tr(dt, arp)
    I32 = np.float32(I0)
    kstar = math.floor(-tau * math.log(1.0 - 1.0 / (R * float(I32))) / dt) + 1
    k_arrive = kstar + TR
    beta = math.exp(-dt / tau)
    tie = (1.0 - beta) * R * float(np.float32(w))
    I = np.zeros((1, 2, k_arrive), np.float32)
    I[0, 0] = I32
    W = np.zeros((2, 2), np.float32)
    W[1, 0] = np.float32(w)
    out = ref.forward_recurrent(I, W, _params(2, tau, 500.0, [1.0, tie], 0.0, R), dt, arp)
    assert int(np.flatnonzero(out.S[0, 0])[0]) + 1 == kstar
    assert out.V[0, 1, -1] == tie and out.theta[0, 1, -1] == tie
    assert out.S[0, 1].sum() == 0
