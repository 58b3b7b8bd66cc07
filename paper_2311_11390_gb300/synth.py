"""Seeded synthetic workloads (inputs only; none of the method's arithmetic).

Each generator draws, with numpy's PCG64 `default_rng(seed)`, the inputs of
one workload of the paper's kind: per-neuron parameters, input currents, or
Poisson input spike rasters.  The paper's datasets (N-MNIST, SHD, Allen V1
recordings) are not available, so these stand in for them:

* `population`      - one ALIF population driven by bias + white noise
                      (B=8, N=128, T=1000, DT=0.1 ms, ARP=2 ms).
* `feedforward`     - Poisson input channels (the synthetic spike dataset of
                      the Supplementary "Speed benchmarks") through dense
                      weights into N ALIF neurons.
* `classification`  - 700-channel rasters with class-dependent rate profiles
                      (stand-in for SHD: 700 channels, 20 classes).
* `neuron_fit`      - 1024 candidate parameter sets driven by one shared
                      Ornstein-Uhlenbeck current (stand-in for the Allen
                      current-clamp recordings).

Spike rasters are returned unpacked (bool [B, C, T]); `pack_bits` gives the
bit-packed layout used by the kernels (bit t%32 of word t//32, LSB first).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class NeuronParams:
    tau_mem: np.ndarray     # [N] ms
    tau_adapt: np.ndarray   # [N] ms
    theta0: np.ndarray      # [N]
    d: np.ndarray           # [N] adaptation scale (the paper's d)
    R: np.ndarray           # [N] input resistance (1 = the paper's normalised form)

    @property
    def N(self):
        return self.tau_mem.shape[0]

    def astype32(self):
        c = lambda x: np.ascontiguousarray(x, dtype=np.float32)
        return NeuronParams(c(self.tau_mem), c(self.tau_adapt), c(self.theta0), c(self.d), c(self.R))


def pack_bits(S: np.ndarray) -> np.ndarray:
    """bool/uint8 [..., T] -> uint32 [..., ceil(T/32)], bit t%32 of word t//32 (LSB first)."""
    S = np.asarray(S).astype(bool)
    T = S.shape[-1]
    W = (T + 31) // 32
    pad = W * 32 - T
    if pad:
        S = np.concatenate([S, np.zeros(S.shape[:-1] + (pad,), bool)], axis=-1)
    by = np.packbits(S.reshape(S.shape[:-1] + (W * 4, 8)), axis=-1, bitorder="little")
    return np.ascontiguousarray(by.reshape(S.shape[:-1] + (W * 4,))).view("<u4").reshape(
        S.shape[:-1] + (W,))


def unpack_bits(words: np.ndarray, T: int) -> np.ndarray:
    """uint32 [..., W] -> uint8 [..., T] (inverse of pack_bits)."""
    words = np.ascontiguousarray(words, dtype="<u4")
    by = words.view(np.uint8).reshape(words.shape[:-1] + (words.shape[-1] * 4, 1))
    bits = np.unpackbits(by, axis=-1, bitorder="little").reshape(words.shape[:-1] + (-1,))
    return bits[..., :T]


def uniform_params(rng, N, tau_mem, tau_adapt, theta0, d, R=1.0) -> NeuronParams:
    """Each argument is a scalar (shared) or a (lo, hi) pair drawn U[lo, hi] per neuron."""
    def draw(v):
        if isinstance(v, tuple):
            return rng.uniform(v[0], v[1], size=N)
        return np.full(N, float(v))
    # fixed draw order: tau_mem, tau_adapt, theta0, d, R
    return NeuronParams(draw(tau_mem), draw(tau_adapt), draw(theta0), draw(d), draw(R)).astype32()


@dataclass
class PopulationWorkload:
    I: np.ndarray           # float32 [B, N, T]
    params: NeuronParams
    dt: float
    arp: float


def population(seed=0, B=8, N=128, T=1000, dt=0.1, arp=2.0, tau_mem=20.0, tau_adapt=200.0,
               theta0=1.0, d=0.1, R=1.0, bias=(0.8, 1.6), noise=0.3) -> PopulationWorkload:
    """I[b,i,t] = bias_i + xi[b,i,t]; bias_i ~ U[bias] shared over the batch, xi ~ N(0, noise^2)."""
    rng = np.random.default_rng(seed)
    params = uniform_params(rng, N, tau_mem, tau_adapt, theta0, d, R)
    b = rng.uniform(bias[0], bias[1], size=N)
    xi = rng.standard_normal((B, N, T), dtype=np.float32) * np.float32(noise)
    I = (b.astype(np.float32)[None, :, None] + xi).astype(np.float32)
    return PopulationWorkload(np.ascontiguousarray(I), params, dt, arp)


@dataclass
class FeedforwardWorkload:
    S_in: np.ndarray        # bool [B, Nin, T]
    W: np.ndarray           # float32 [N, Nin]
    bias: np.ndarray        # float32 [N]
    params: NeuronParams
    dt: float
    arp: float


def poisson_raster(rng, B, C, T, rates_hz, dt_ms) -> np.ndarray:
    """Bernoulli(rate_c * DT) per (b, c, t); rates_hz: [C] (or [B, C]).  bool [B, C, T]."""
    prob = np.broadcast_to(np.asarray(rates_hz, np.float64) * dt_ms * 1e-3, (B, C)).astype(np.float32)
    out = np.empty((B, C, T), dtype=bool)
    for b in range(B):
        out[b] = rng.random((C, T), dtype=np.float32) < prob[b][:, None]
    return out


def feedforward(seed=0, B=32, Nin=1000, N=1024, T=1000, dt=0.1, arp=2.0, rates=(10.0, 50.0),
                w_std=None, bias=(0.8, 1.6), tau_mem=(10.0, 30.0), tau_adapt=(100.0, 500.0),
                theta0=1.0, d=(0.0, 0.2), R=1.0) -> FeedforwardWorkload:
    """Poisson channels (rates U[rates] per channel) -> W ~ N(0, 2/Nin) -> N ALIF neurons
    with bias_i ~ U[bias] (the paper's b_i of Eq 3)."""
    rng = np.random.default_rng(seed)
    params = uniform_params(rng, N, tau_mem, tau_adapt, theta0, d, R)
    std = np.sqrt(2.0 / Nin) if w_std is None else w_std
    W = (rng.standard_normal((N, Nin)) * std).astype(np.float32)
    b = rng.uniform(bias[0], bias[1], size=N).astype(np.float32)
    r = rng.uniform(rates[0], rates[1], size=Nin)
    S = poisson_raster(rng, B, Nin, T, r, dt)
    return FeedforwardWorkload(S, W, b, params, dt, arp)


@dataclass
class ClassificationWorkload:
    S_in: np.ndarray        # bool [B, 700, T]
    labels: np.ndarray      # int64 [B]
    W: list                 # [W1 [256,700], W2 [256,256], Wout [20,256]] float32
    bias: list              # [b1 [256], b2 [256]] float32
    params: list            # NeuronParams for the two hidden layers
    tau_out: float          # readout membrane time constant (ms)
    dt: float
    arp: float


def classification(seed=0, B=128, T=1000, dt=1.0, arp=2.0, channels=700, classes=20,
                   hidden=(256, 256), bias=(0.8, 1.6)) -> ClassificationWorkload:
    """Class c has channel rate profile r_j = 5 + 45 exp(-(j - mu_c)^2 / (2 * 50^2)) Hz with
    mu_c = 35 c + 17; weights U(+-1/sqrt(fan_in)); tau_mem 20, tau_adapt 150, d 1.8 (the
    Supplementary's classification initialisation); hidden bias U[bias]."""
    rng = np.random.default_rng(seed)
    labels = rng.integers(0, classes, size=B)
    j = np.arange(channels)
    mu = 35.0 * labels + 17.0
    rates = 5.0 + 45.0 * np.exp(-((j[None, :] - mu[:, None]) ** 2) / (2 * 50.0 ** 2))
    S = poisson_raster(rng, B, channels, T, rates, dt)
    sizes = [channels, *hidden, classes]
    Ws = []
    for fan_in, fan_out in zip(sizes[:-1], sizes[1:]):
        lim = 1.0 / np.sqrt(fan_in)
        Ws.append(rng.uniform(-lim, lim, size=(fan_out, fan_in)).astype(np.float32))
    bs = [rng.uniform(bias[0], bias[1], size=h).astype(np.float32) for h in hidden]
    ps = [uniform_params(rng, h, 20.0, 150.0, 1.0, 1.8) for h in hidden]
    return ClassificationWorkload(S, labels.astype(np.int64), Ws, bs, ps, 20.0, dt, arp)


@dataclass
class FitWorkload:
    I: np.ndarray           # float32 [1, N, T] (the same OU current for every candidate)
    params: NeuronParams    # N candidate parameter sets
    hidden: NeuronParams    # the 1-neuron parameter set that makes the target train
    dt: float
    arp: float
    tau_vr: float           # van Rossum kernel time constant (ms)


def ou_current(rng, T, dt, tau=3.0, mean=0.5, sigma=0.5) -> np.ndarray:
    """Exact Ornstein-Uhlenbeck update x <- x e^{-DT/tau} + mean (1 - e^{-DT/tau})
    + sigma sqrt(1 - e^{-2 DT/tau}) xi, started from the stationary law.  float32 [T]."""
    e = np.exp(-dt / tau)
    s = sigma * np.sqrt(1.0 - e * e)
    xi = rng.standard_normal(T)
    x = np.empty(T)
    v = mean + sigma * rng.standard_normal()
    for t in range(T):
        v = v * e + mean * (1.0 - e) + s * xi[t]
        x[t] = v
    return x.astype(np.float32)


def neuron_fit(seed=0, N=1024, T=400000, dt=0.05, arp=2.0, tau_vr=5.0) -> FitWorkload:
    rng = np.random.default_rng(seed)
    params = uniform_params(rng, N, (5.0, 40.0), (50.0, 1000.0), (0.5, 2.0), (0.0, 0.5), (0.5, 2.0))
    hidden = NeuronParams(*(np.array([v], np.float32) for v in (20.0, 200.0, 1.0, 0.1, 1.5)))
    x = ou_current(rng, T, dt)
    I = np.ascontiguousarray(np.broadcast_to(x[None, None, :], (1, N, T)))
    return FitWorkload(I, params, hidden, dt, arp, tau_vr)


@dataclass
class DtSweepWorkload:
    params: NeuronParams    # [n] fit-like parameter sets
    x_fine: np.ndarray      # float32 [T_fine] one OU current on the fine grid
    fine_dt: float          # ms
    seconds: float


def dt_sweep(seed=21, n=1024, seconds=1.0, fine_dt=0.01) -> DtSweepWorkload:
    """Speed-accuracy sweep over DT (the trade-off of the paper's opening figure): n neurons with
    fit-like parameters (tau_mem U[5,40] ms, tau_adapt U[50,1000] ms, theta0 U[0.5,2], d U[0,0.5],
    R U[0.5,2]) driven by one Ornstein-Uhlenbeck current (tau 3 ms, mean 0.5, sigma 0.5) drawn
    on the fine grid for `seconds`."""
    rng = np.random.default_rng(seed)
    p = uniform_params(rng, n, (5.0, 40.0), (50.0, 1000.0), (0.5, 2.0), (0.0, 0.5), (0.5, 2.0))
    T = int(round(seconds * 1e3 / fine_dt))
    return DtSweepWorkload(p, ou_current(rng, T, fine_dt), fine_dt, seconds)


def bin_current(x_fine: np.ndarray, f: int) -> np.ndarray:
    """The fine current averaged over bins of f steps (the input a coarse-DT run sees), float32."""
    T = x_fine.shape[-1] // f
    return x_fine[..., : T * f].astype(np.float64).reshape(*x_fine.shape[:-1], T, f).mean(-1).astype(np.float32)


def place_on_fine_grid(S: np.ndarray, f: int) -> np.ndarray:
    """Coarse spike trains [..., T] -> the fine grid [..., T f], each spike at the end of its bin."""
    out = np.zeros(S.shape[:-1] + (S.shape[-1] * f,), np.uint8)
    out[..., f - 1::f] = S
    return out
