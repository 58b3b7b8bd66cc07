"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Every check here is independent of the oracle's own code: closed forms, a
library routine, exact rational arithmetic, brute force over all spike
trains, and the paper's blocked reformulation (Section 3, Props 1-5) written
out separately.  A plausible slip in the oracle (a dropped reset, an
off-by-one in the refractory counter, a wrong adaptation index, ">=" for ">")
fails at least one of them.
"""
import math
from fractions import Fraction as F

import numpy as np
import pytest
import scipy.signal

from oracle import exact
from paper_2311_11390_gb300 import synth


def _params(N, tau_mem, tau_adapt, theta0, d, R=1.0):
    from oracle.ref import Params
    f = lambda v: np.full(N, v, np.float64) if np.isscalar(v) else np.asarray(v, np.float64)
    return Params(f(tau_mem), f(tau_adapt), f(theta0), f(d), f(R))


# ---------------------------------------------------------------- T_R ------
def test_tr_rounding(oracle_lib):
    ref = oracle_lib
    assert ref.tr(0.1, 2.0) == 20          # 2/0.1 is not exact in binary
    assert ref.tr(0.05, 2.0) == 40
    assert ref.tr(1.0, 2.0) == 2
    assert ref.tr(0.1, 0.1) == 1
    assert ref.tr(0.3, 1.0) == -1          # not an integer number of steps
    assert ref.tr(0.1, 0.05) == -1         # shorter than one step
    assert ref.tr(0.0, 2.0) == -1


# ------------------------------------------------- LIF closed form (d = 0) --
LIF_CASES = [
    # tau_mem, dt, theta0, R, I, arp
    (20.0, 0.1, 1.0, 1.0, 1.37, 2.0),
    (10.0, 0.1, 1.0, 1.5, 0.9, 1.0),
    (5.0, 1.0, 0.7, 1.0, 2.3, 2.0),
    (30.0, 0.05, 1.2, 2.0, 0.77, 2.0),
    (20.0, 0.1, 1.0, 1.0, 5.0, 0.1),       # T_R = 1 behaves like T_R = 2 (reset kills t+1)
]


@pytest.mark.parametrize("tau, dt, th0, R, I0, arp", LIF_CASES)
def test_lif_first_passage_closed_form(oracle_lib, tau, dt, th0, R, I0, arp):
    """d = 0, constant drive from rest: V[k] = R I (1 - beta^k) and the first spike is at
    k* = floor(t*/DT) + 1 with t* = -tau ln(1 - theta0/(R I)); later ISIs are max(T_R,2) - 1 + k*
    (reset zeroes V at the next step, the ARP holds the input off until C >= T_R)."""
    ref = oracle_lib
    TR = ref.tr(dt, arp)
    I32 = np.float32(I0)
    RI = R * float(I32)
    tstar = -tau * math.log(1.0 - th0 / RI)
    ratio = tstar / dt
    assert abs(ratio - round(ratio)) > 1e-6, "case too close to an integer crossing"
    kstar = math.floor(ratio) + 1
    isi = max(TR, 2) - 1 + kstar
    T = kstar + 4 * isi + 3
    I = np.full((1, 1, T), I32, np.float32)
    out = ref.forward(I, _params(1, tau, 500.0, th0, 0.0, R), dt, arp)
    spikes = np.flatnonzero(out.S[0, 0]) + 1   # paper time
    expected = [kstar + n * isi for n in range(T) if kstar + n * isi <= T]
    assert spikes.tolist() == expected
    beta = math.exp(-dt / tau)
    k = np.arange(1, kstar + 1)
    np.testing.assert_allclose(out.V[0, 0, :kstar], RI * (1 - beta ** k), rtol=1e-13, atol=1e-15)
    # refractory: V = 0 from the step after the spike until input is admitted again
    s0 = kstar
    assert np.all(out.V[0, 0, s0: s0 + max(TR, 2) - 1] == 0.0)


def test_strict_threshold_at_exact_tie(oracle_lib):
    """Eq 1 is strict (V > theta): a neuron held exactly at threshold never fires.  With
    V[0] = theta0 = 1, d = 0, R = 1 and I = 1, beta*1 + (1-beta)*1 is exactly 1 in binary
    floating point (1 - beta is exact for beta in [1/2, 1)), so V stays exactly on theta."""
    ref = oracle_lib
    T = 500
    I = np.ones((1, 2, T), np.float32)
    I[0, 1] = np.float32(1.0 + 2.0 ** -20)       # a hair above: fires
    out = ref.forward(I, _params(2, 20.0, 200.0, 1.0, 0.0), 0.1, 2.0,
                      init=ref.Init(V=np.array([1.0, 1.0])))
    assert np.all(out.V[0, 0] == 1.0)
    assert out.S[0, 0].sum() == 0
    assert out.S[0, 1].sum() > 0


# ------------------------------------------------ library-routine special case
def test_no_spike_membrane_is_linear_filter(oracle_lib):
    """Threshold out of reach: no spikes, V is the unrolled Eq 2 (Prop 1 / its proof):
    V[t] = beta^t V[0] + (1-beta) sum_j beta^{t-j} R I[j]; a[t] = p^t a[0]."""
    ref = oracle_lib
    rng = np.random.default_rng(3)
    B, N, T = 2, 3, 400
    I = rng.normal(0.3, 1.0, size=(B, N, T)).astype(np.float32)
    tm = np.array([5.0, 20.0, 80.0]); ta = np.array([50.0, 200.0, 900.0])
    R = np.array([0.5, 1.0, 2.0])
    par = _params(N, tm, ta, 1e6, 0.3, R)
    V0 = rng.normal(size=B * N); a0 = rng.uniform(0, 2, size=B * N)
    out = ref.forward(I, par, 0.1, 2.0, init=ref.Init(V=V0, a=a0))
    assert out.S.sum() == 0
    for b in range(B):
        for i in range(N):
            beta = math.exp(-0.1 / tm[i]); p = math.exp(-0.1 / ta[i])
            x = R[i] * I[b, i].astype(np.float64)
            zi = scipy.signal.lfiltic([1 - beta], [1, -beta], y=[V0[b * N + i]])
            V, _ = scipy.signal.lfilter([1 - beta], [1, -beta], x, zi=zi)
            np.testing.assert_allclose(out.V[b, i], V, rtol=1e-11, atol=1e-12)
            np.testing.assert_allclose(out.a[b, i], p ** np.arange(1, T + 1) * a0[b * N + i],
                                       rtol=1e-11, atol=1e-300)


# ----------------------------------------------- reduction to LIF (d = 0) ---
def _lif_loop(I, beta, th0, TR, R):
    """Independent textbook discrete LIF with reset and absolute refractory period."""
    V, out_S, out_V, last = 0.0, [], [], None
    for t, x in enumerate(I):
        if last is not None and t == last + 1:
            V = 0.0                                          # reset
        elif last is None or t - last >= TR:
            V = beta * V + (1 - beta) * R * float(x)
        else:
            V = beta * V                                     # refractory: no input
        s = V > th0
        if s:
            last = t
        out_S.append(int(s)); out_V.append(V)
    return np.array(out_S), np.array(out_V)


@pytest.mark.parametrize("seed", [0, 1])
def test_reduces_to_lif_when_d_is_zero(oracle_lib, seed):
    ref = oracle_lib
    w = synth.population(seed=seed, B=2, N=16, T=600, d=0.0)
    out = ref.forward(w.I, _params(16, w.params.tau_mem, w.params.tau_adapt, w.params.theta0,
                                   0.0, w.params.R), w.dt, w.arp)
    TR = ref.tr(w.dt, w.arp)
    assert out.S.sum() > 20
    for b in range(2):
        for i in range(16):
            beta = math.exp(-w.dt / float(w.params.tau_mem[i]))
            S, V = _lif_loop(w.I[b, i], beta, float(w.params.theta0[i]), TR, float(w.params.R[i]))
            assert np.array_equal(S, out.S[b, i])
            np.testing.assert_allclose(V, out.V[b, i], rtol=1e-12, atol=1e-14)


# --------------------------------------------- exact arithmetic, brute force -
def _exact_case(rng, T):
    beta = F(rng.integers(1, 9), 10); p = F(rng.integers(1, 10), 10)
    theta0 = F(rng.integers(5, 12), 10); d = F(rng.integers(0, 8), 10)
    TR = int(rng.integers(1, 5))
    I = [F(int(v), 4) for v in rng.integers(-2, 12, size=T)]
    return beta, p, theta0, d, TR, I


@pytest.mark.parametrize("seed", range(6))
def test_brute_force_unique_consistent_train(seed):
    """Eqs 1-5 define the spike train as the unique self-consistent one: among all 2^T
    trains exactly one satisfies S = 1{V > theta} with V, a driven by S itself."""
    rng = np.random.default_rng(100 + seed)
    T = 10 if seed < 4 else 12
    beta, p, theta0, d, TR, I = _exact_case(rng, T)
    sols = exact.brute_force(I, beta, p, theta0, d, TR)
    assert len(sols) == 1
    S, _, _, _ = exact.simulate(I, beta, p, theta0, d, TR)
    assert sols[0] == S


@pytest.mark.parametrize("seed", range(8))
def test_oracle_matches_exact_rational(oracle_lib, seed):
    """FP64 oracle vs exact rational simulation on the oracle's own (exactly representable)
    coefficients: same spikes, traces to 1e-12."""
    ref = oracle_lib
    rng = np.random.default_rng(200 + seed)
    T = 48
    dt = 0.1
    tm = float(rng.uniform(0.5, 30)); ta = float(rng.uniform(0.5, 300))
    th0 = float(np.float32(rng.uniform(0.3, 1.5))); d = float(np.float32(rng.uniform(0, 1)))
    R = float(np.float32(rng.uniform(0.5, 2)))
    arp = [0.1, 0.2, 0.4, 0.7][seed % 4]
    TR = ref.tr(dt, arp)
    I = rng.normal(1.2, 1.0, size=(1, 1, T)).astype(np.float32)
    out = ref.forward(I, _params(1, tm, ta, th0, d, R), dt, arp)
    beta = F(math.exp(-dt / tm)); p = F(math.exp(-dt / ta))
    S, V, a, th = exact.simulate([F(float(x)) for x in I[0, 0]], beta, p, F(th0), F(d), TR, R=F(R))
    margins = [abs(float(v - t)) for v, t in zip(V, th)]
    assert min(margins) > 1e-9, "tie in the random case"
    assert out.S[0, 0].tolist() == S
    np.testing.assert_allclose(out.V[0, 0], [float(v) for v in V], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(out.a[0, 0], [float(v) for v in a], rtol=1e-12, atol=1e-14)


# ------------------------------------------ the paper's blocked reformulation
def _blocks(I, beta, p, th0, d, R, TR):
    """Section 3 written out: Blocks of T_R steps.  Inside a block the no-reset membrane is
    the convolution of Prop 1 (initial potential folded in as I[0] = V[0]/(1-beta)), faulty
    spikes S~ = f(V~), latent timing z = phi(S~) (Prop 2), correct spikes S = 1{z = 1};
    across blocks the input mask of Prop 3, the membrane carry of Prop 4 and the
    adaptation carry of Prop 5.  Zero padding to a multiple of T_R (footnote, Section 3.2)."""
    T = len(I)
    nb = -(-T // TR)
    x = np.zeros(nb * TR); x[:T] = R * np.asarray(I, np.float64)
    t = np.arange(1, TR + 1)
    K = np.tril(beta ** (t[:, None] - t[None, :]))          # beta^{t-j}, j <= t
    S_all = np.zeros(nb * TR, np.int64)
    V0, a0 = 0.0, 0.0
    z_prev, S_prev = np.zeros(TR), np.zeros(TR)
    for n in range(nb):
        blk = x[n * TR:(n + 1) * TR]
        mask = (z_prev >= S_prev.max()).astype(np.float64)   # Prop 3 (ARP mask)
        Vt = beta ** t * V0 + (1 - beta) * (K @ (blk * mask))  # Prop 1
        theta = th0 + d * p ** t * a0                          # Prop 5
        St = (Vt > theta).astype(np.int64)                     # Eq 7
        z = np.cumsum(np.cumsum(St))                           # Prop 2: phi
        S = (z == 1).astype(np.int64)                          # Eq 9
        if S.any():
            ts = int(np.argmax(S)) + 1
            m = TR - ts
            a_s = p ** ts * a0                                 # a at the spike
            a0 = p ** m * (a_s + 1.0 / p)                      # Prop 5, spiked
            V0 = 0.0                                           # Prop 4, spiked
        else:
            a0 = p ** TR * a0                                  # Prop 5, no spike
            V0 = Vt[-1]                                        # Prop 4, no spike
        S_all[n * TR:(n + 1) * TR] = S
        z_prev, S_prev = z, S
    return S_all[:T]


@pytest.mark.parametrize("seed, arp", [(0, 2.0), (1, 1.0), (2, 4.0), (3, 0.3)])
def test_oracle_equals_paper_blocks(oracle_lib, seed, arp):
    """Props 1-5 ('mathematically the same', Section 3): the blocked form reproduces the
    oracle's spike trains exactly, except at FP64 near-ties (none expected here)."""
    ref = oracle_lib
    w = synth.population(seed=seed, B=2, N=24, T=997, arp=arp,
                         tau_adapt=(60.0, 300.0), d=(0.0, 0.6))
    out = ref.forward(w.I, ref.Params(*w.params.astype32().__dict__.values()), w.dt, w.arp)
    TR = ref.tr(w.dt, w.arp)
    assert out.S.sum() > 50
    assert np.abs(out.margin).min() > 1e-9
    for b in range(2):
        for i in range(24):
            beta = math.exp(-w.dt / float(w.params.tau_mem[i]))
            p = math.exp(-w.dt / float(w.params.tau_adapt[i]))
            S = _blocks(w.I[b, i], beta, p, float(w.params.theta0[i]), float(w.params.d[i]),
                        float(w.params.R[i]), TR)
            assert np.array_equal(S, out.S[b, i]), (b, i)


def test_phi_prop2_example():
    """Prop 2: phi maps the first faulty spike to 1 and every later step to > 1 (hand-evaluated)."""
    assert exact.phi([0, 0, 1, 0, 1, 1]) == [0, 0, 1, 2, 4, 7]
    assert exact.phi([0, 0, 0]) == [0, 0, 0]


# ---------------------------------------------------------------- invariants -
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_arp_invariants(oracle_lib, seed):
    """At most one spike in any T_R consecutive steps (Fig 1c); V = 0 on the T_R - 1 steps
    after a spike; a[t+1] - p a[t] = S[t] (Eq 5); Prop 5's carry
    a_{n}[T_R] = p^m (a_s + 1/p) for every block with a spike; and Prop 3's mask count:
    steps masked at the start of block n+1 = t_s - 1 of block n."""
    ref = oracle_lib
    w = synth.population(seed=seed, B=4, N=32, T=1000, tau_adapt=(80.0, 400.0), d=(0.05, 0.5))
    out = ref.forward(w.I, ref.Params(*w.params.astype32().__dict__.values()), w.dt, w.arp)
    TR = ref.tr(w.dt, w.arp)
    S = out.S.astype(np.int64)
    assert S.sum() > 100
    win = np.lib.stride_tricks.sliding_window_view(S, TR, axis=-1).sum(-1)
    assert win.max() == 1
    for b, i, k in zip(*np.nonzero(S)):
        assert np.all(out.V[b, i, k + 1:k + TR] == 0.0)
    p = np.exp(-w.dt / w.params.tau_adapt.astype(np.float64))[None, :, None]
    np.testing.assert_allclose(out.a[:, :, 1:] - p * out.a[:, :, :-1], S[:, :, :-1], atol=1e-12)
    nb = 1000 // TR
    Sb = S[:, :, :nb * TR].reshape(4, 32, nb, TR)
    ab = out.a[:, :, :nb * TR].reshape(4, 32, nb, TR)
    mb = out.mask[:, :, :nb * TR].reshape(4, 32, nb, TR)
    checked = 0
    for b, i, n in zip(*np.nonzero(Sb.sum(-1))):
        if n + 1 >= nb:
            continue
        ts = int(np.argmax(Sb[b, i, n])) + 1
        m = TR - ts
        pi = float(p[0, i, 0])
        a_s = ab[b, i, n, ts - 1]
        # Prop 5: theta_{n+1}[t] = theta0 + d p^t a_{n+1}[0], a_{n+1}[0] = p^m (a_s + 1/p)
        np.testing.assert_allclose(ab[b, i, n + 1, 0], pi * pi ** m * (a_s + 1.0 / pi), rtol=1e-12)
        # Prop 3: the first t_s - 1 steps of block n+1 are masked, the rest admitted
        assert np.all(mb[b, i, n + 1, :ts - 1] == 0) and np.all(mb[b, i, n + 1, ts - 1:] == 1)
        checked += 1
    assert checked > 60


# ---------------------------------------------------- adaptation fixed point -
def test_adaptive_fixed_point(oracle_lib):
    """Constant drive with d > 0: inter-spike intervals never shrink and settle; at the settled
    interval D the post-spike adaptation is the geometric series a* = 1/(1 - p^D)."""
    ref = oracle_lib
    T = 40000
    I = np.full((1, 1, T), np.float32(1.8), np.float32)
    out = ref.forward(I, _params(1, 20.0, 20.0, 1.0, 0.4), 0.1, 2.0)
    sp = np.flatnonzero(out.S[0, 0])
    isi = np.diff(sp)
    assert len(isi) > 30
    assert np.all(np.diff(isi) >= 0) or np.all(np.diff(isi[len(isi) // 2:]) == 0)
    D = int(isi[-1])
    assert np.all(isi[-10:] == D)
    p = math.exp(-0.1 / 20.0)
    a_after = out.a[0, 0, sp[-2] + 1]     # a one step after a spike (includes the jump)
    np.testing.assert_allclose(a_after, 1.0 / (1.0 - p ** D), rtol=1e-9)


# ------------------------------------------------------------ backward pins --
def _torch_bptt(I, tm, ta, th0, d, R, dt, TR, gS, gV, ga, slope, surrogate="fast_sigmoid",
                attached=False):
    """float64 autograd through a plain step loop (spike: Heaviside forward, surrogate
    backward; S detached in the reset and the adaptation update unless `attached`; the ARP
    mask is data).  The multi-Gaussian surrogate is built from torch's normal distribution
    densities."""
    import torch

    def sg(u):
        if surrogate == "multi_gaussian":
            N = torch.distributions.Normal
            dens = lambda mu, sd: N(torch.tensor(mu, dtype=u.dtype), torch.tensor(sd, dtype=u.dtype)).log_prob(u).exp()
            return 1.15 * dens(0.0, 0.5) - 0.15 * dens(3.0, 3.0) - 0.15 * dens(-3.0, 3.0)
        if surrogate == "boxcar":
            return torch.where(u.abs() <= 0.5, torch.full_like(u, 0.5), torch.zeros_like(u))
        return 1.0 / (slope * u.abs() + 1.0) ** 2

    class Spike(torch.autograd.Function):
        @staticmethod
        def forward(ctx, u):
            ctx.save_for_backward(u)
            return (u > 0).to(u.dtype)

        @staticmethod
        def backward(ctx, g):
            (u,) = ctx.saved_tensors
            return g * sg(u)

    f = lambda v: torch.tensor(v, dtype=torch.float64, requires_grad=True)
    tm, ta, th0, d, R = f(tm), f(ta), f(th0), f(d), f(R)
    Ix = torch.tensor(I.astype(np.float64), requires_grad=True)
    gS, gV, ga = (torch.as_tensor(np.asarray(g, np.float64)) for g in (gS, gV, ga))
    beta = torch.exp(-dt / tm); p = torch.exp(-dt / ta)
    V = torch.zeros(I.shape[:-1], dtype=torch.float64)
    a = torch.zeros_like(V); S = torch.zeros_like(V)
    last = torch.full(V.shape, -10 ** 9, dtype=torch.int64)
    loss = 0.0
    for k in range(I.shape[-1]):
        Sg = S if attached else S.detach()
        a = p * a + Sg
        th = th0 + d * a
        m = ((k - last) >= TR).to(torch.float64)
        V = (beta * V + (1 - beta) * m * R * Ix[..., k]) * (1 - Sg)
        S = Spike.apply(V - th)
        last = torch.where(S > 0, torch.full_like(last, k), last)
        loss = loss + (S * gS[..., k]).sum() + (V * gV[..., k]).sum() + (a * ga[..., k]).sum()
    loss.backward()
    return Ix.grad.numpy(), [x.grad.numpy() for x in (tm, ta, th0, d, R)]


@pytest.mark.parametrize("seed, arp", [(0, 1.5), (1, 1.5), (2, 0.5)])
def test_backward_matches_autograd(oracle_lib, seed, arp):
    """Hand BPTT of the oracle vs float64 autograd (T_R = 3 and T_R = 1)."""
    ref = oracle_lib
    rng = np.random.default_rng(seed)
    N, T = 3, 160
    I = (1.3 + 0.4 * rng.standard_normal((1, N, T))).astype(np.float32)
    tm = rng.uniform(2, 10, N); ta = rng.uniform(20, 80, N)
    th0 = rng.uniform(0.8, 1.2, N); d = rng.uniform(0.1, 0.5, N); R = rng.uniform(0.8, 1.5, N)
    gS = rng.standard_normal((1, N, T)); gV = rng.standard_normal((1, N, T))
    ga = rng.standard_normal((1, N, T))
    dt, slope = 0.5, 25.0
    TR = ref.tr(dt, arp)
    out = ref.forward(I, _params(N, tm, ta, th0, d, R), dt, arp)
    assert out.S.sum() >= 6
    bw = ref.backward(I, _params(N, tm, ta, th0, d, R), dt, arp, gS, gV, ga, slope=slope)
    gI_t, (g_tm, g_ta, g_th0, g_d, g_R) = _torch_bptt(I[0], tm, ta, th0, d, R, dt, TR,
                                                      gS[0], gV[0], ga[0], slope)
    np.testing.assert_allclose(bw.gI[0], gI_t, rtol=1e-9, atol=1e-12)
    for mine, theirs in [(bw.g_tau_mem, g_tm), (bw.g_tau_adapt, g_ta), (bw.g_theta0, g_th0),
                         (bw.g_d, g_d), (bw.g_R, g_R)]:
        np.testing.assert_allclose(mine[0], theirs, rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("surrogate", ["multi_gaussian", "boxcar"])
def test_backward_surrogates_match_autograd(oracle_lib, surrogate):
    """The other surrogates of the Supplementary's comparison: the oracle's BPTT with the
    multi-Gaussian (as printed: means 0 and +-3, standard deviations 0.5 and 3) and the boxcar
    (0.5 within |V - theta| <= 0.5) against float64 autograd built on the same definitions."""
    ref = oracle_lib
    rng = np.random.default_rng(4)
    N, T = 3, 160
    I = (1.3 + 0.4 * rng.standard_normal((1, N, T))).astype(np.float32)
    tm = rng.uniform(2, 10, N); ta = rng.uniform(20, 80, N)
    th0 = rng.uniform(0.8, 1.2, N); d = rng.uniform(0.1, 0.5, N); R = rng.uniform(0.8, 1.5, N)
    gS = rng.standard_normal((1, N, T)); gV = rng.standard_normal((1, N, T))
    ga = rng.standard_normal((1, N, T))
    dt, arp = 0.5, 1.5
    TR = ref.tr(dt, arp)
    bw = ref.backward(I, _params(N, tm, ta, th0, d, R), dt, arp, gS, gV, ga, surrogate=surrogate)
    gI_t, (g_tm, g_ta, g_th0, g_d, g_R) = _torch_bptt(I[0], tm, ta, th0, d, R, dt, TR,
                                                      gS[0], gV[0], ga[0], 25.0, surrogate)
    np.testing.assert_allclose(bw.gI[0], gI_t, rtol=1e-9, atol=1e-12)
    for mine, theirs in [(bw.g_tau_mem, g_tm), (bw.g_tau_adapt, g_ta), (bw.g_theta0, g_th0),
                         (bw.g_d, g_d), (bw.g_R, g_R)]:
        np.testing.assert_allclose(mine[0], theirs, rtol=1e-9, atol=1e-12)
    # the surrogate reached theta0: its gradient is not identically zero
    assert np.abs(bw.g_theta0).max() > 1e-6


@pytest.mark.parametrize("surrogate, arp", [("fast_sigmoid", 1.5), ("fast_sigmoid", 0.5),
                                             ("multi_gaussian", 1.5), ("boxcar", 1.0)])
def test_backward_attached_matches_autograd(oracle_lib, surrogate, arp):
    """"Attached" gradients (Supplementary, "Detaching gradients"): S[t] keeps its surrogate
    gradient in the reset factor of V[t+1] and in the update of a[t+1].  The oracle's hand
    BPTT against float64 autograd over the same step loop without the detaches (T_R = 3, 1
    and 2); and it differs from the detached gradient."""
    ref = oracle_lib
    rng = np.random.default_rng(11)
    N, T = 3, 160
    I = (1.3 + 0.4 * rng.standard_normal((1, N, T))).astype(np.float32)
    tm = rng.uniform(2, 10, N); ta = rng.uniform(20, 80, N)
    th0 = rng.uniform(0.8, 1.2, N); d = rng.uniform(0.1, 0.5, N); R = rng.uniform(0.8, 1.5, N)
    gS = rng.standard_normal((1, N, T)); gV = rng.standard_normal((1, N, T))
    ga = rng.standard_normal((1, N, T))
    dt, slope = 0.5, 5.0
    TR = ref.tr(dt, arp)
    P = _params(N, tm, ta, th0, d, R)
    assert ref.forward(I, P, dt, arp).S.sum() >= 6
    bw = ref.backward(I, P, dt, arp, gS, gV, ga, slope=slope, surrogate=surrogate, attached=True)
    gI_t, (g_tm, g_ta, g_th0, g_d, g_R) = _torch_bptt(I[0], tm, ta, th0, d, R, dt, TR,
                                                      gS[0], gV[0], ga[0], slope, surrogate, attached=True)
    np.testing.assert_allclose(bw.gI[0], gI_t, rtol=1e-9, atol=1e-12)
    for mine, theirs in [(bw.g_tau_mem, g_tm), (bw.g_tau_adapt, g_ta), (bw.g_theta0, g_th0),
                         (bw.g_d, g_d), (bw.g_R, g_R)]:
        np.testing.assert_allclose(mine[0], theirs, rtol=1e-9, atol=1e-12)
    det = ref.backward(I, P, dt, arp, gS, gV, ga, slope=slope, surrogate=surrogate)
    assert np.abs(det.gI - bw.gI).max() > 1e-3 * np.abs(bw.gI).max()


def test_backward_matches_finite_differences(oracle_lib):
    """Loss on the V and a traces only (no spike term): V and a are piecewise smooth in
    I, R, tau_mem, tau_adapt for fixed spike times, so central differences equal the
    analytic gradient as long as no spike moves (checked)."""
    ref = oracle_lib
    rng = np.random.default_rng(7)
    N, T = 2, 300
    I = (1.2 + 0.3 * rng.standard_normal((1, N, T))).astype(np.float64)
    tm = np.array([12.0, 25.0]); ta = np.array([80.0, 300.0])
    th0 = np.array([1.0, 0.9]); d = np.array([0.2, 0.4]); R = np.array([1.1, 0.9])
    wV = rng.standard_normal((1, N, T)); wa = rng.standard_normal((1, N, T))
    dt, arp = 0.1, 2.0

    def run(I_, tm_, ta_, R_):
        o = ref.forward(I_.astype(np.float32), _params(N, tm_, ta_, th0, d, R_), dt, arp)
        return o, float((o.V * wV).sum() + (o.a * wa).sum())

    base, _ = run(I, tm, ta, R)
    bw = ref.backward(I.astype(np.float32), _params(N, tm, ta, th0, d, R), dt, arp,
                      np.zeros((1, N, T)), wV, wa)

    def fd(fun, eps):
        o1, l1 = fun(+eps); o2, l2 = fun(-eps)
        assert np.array_equal(o1.S, base.S) and np.array_equal(o2.S, base.S)
        return (l1 - l2) / (2 * eps)

    for i in range(N):
        for name, g in (("tm", bw.g_tau_mem), ("ta", bw.g_tau_adapt), ("R", bw.g_R)):
            def fun(e, i=i, name=name):
                tm_, ta_, R_ = tm.copy(), ta.copy(), R.copy()
                {"tm": tm_, "ta": ta_, "R": R_}[name][i] += e
                return run(I, tm_, ta_, R_)
            num = fd(fun, 1e-6)
            np.testing.assert_allclose(g[0, i], num, rtol=2e-5, atol=1e-7)
    # current: I is float32 in the oracle, so perturb by exactly representable amounts
    for (i, k) in [(0, 5), (0, 150), (1, 80), (1, 299)]:
        def fun(e, i=i, k=k):
            I2 = I.astype(np.float32).astype(np.float64).copy()
            I2[0, i, k] += e
            return run(I2, tm, ta, R)
        num = fd(fun, 2.0 ** -12)
        np.testing.assert_allclose(bw.gI[0, i, k], num, rtol=1e-5, atol=1e-9)
    assert np.all(bw.g_theta0 == 0) and np.all(bw.g_d == 0)
