"""The lane-per-row forward's margin error bound, checked on the CPU (no GPU).

`fwd_rows_kernel` takes a spike decision in FP32 unless the margin lies within an error bound G,
where it re-decides in double-single.  The decisions are exact only if G really bounds the FP32
margin's error, so G is derived term by term in the kernel's header (Prop 1's no-reset membrane
V~[k] = beta^(k+1) v_in + L[k] over a Block of K steps; the carried double-single membrane; the
effective membrane W = -beta^-r L[r-1] of a Block entered part-way through the ARP):

    G = (1 + 2^-6) (u (4 M + 5 |d a| + theta0) + (4K + 4) u R (1 - beta^K) max_Block|I|
                    + (2K + 4) u R max_row|I|),   M = max(|v_in|, R max_Block|I|),  u = 2^-24.

Here the kernel's FP32 pipeline is restated in NumPy (FP32 products and FMAs, the latter as an
exact FP64 product-sum rounded once to FP32; the double-single carries as FP64), run over Blocks
on the feedforward workload's currents (from the FP64 projection oracle), and each admitted margin
is compared with the same margin in FP64 (the masked membrane of Eq 4 and the threshold of Eq 5).
The bound must hold with room to spare: a margin error above half of G fails.  Spike decisions
follow FP64 (the kernel's re-decisions make them exact), so both sides walk the same spikes.
"""
import numpy as np
import pytest

from oracle import project
from paper_2311_11390_gb300 import synth

f32 = np.float32
U = 2.0 ** -24


def _fma(a, b, c):
    return (np.asarray(a, np.float64) * np.asarray(b, np.float64) + np.asarray(c, np.float64)).astype(f32)


def _mul(a, b):
    return (np.asarray(a, np.float64) * np.asarray(b, np.float64)).astype(f32)


def _margin_errors(K, rows, T, scale, tau_mem, d, seed):
    """Largest |Z - Z*| / G over admitted margins within 1e-3 of threshold, over all admitted
    margins, and the spike count."""
    w = synth.feedforward(seed=seed, B=1, Nin=1000, N=rows, T=T, dt=0.1, arp=2.0, tau_mem=tau_mem, d=d)
    I = (project.project(w.W, w.S_in, w.bias)[0] * scale).astype(f32)
    P = w.params
    beta = np.exp(-w.dt / P.tau_mem.astype(np.float64))
    p = np.exp(-w.dt / P.tau_adapt.astype(np.float64))
    R = P.R.astype(np.float64)
    th0 = P.theta0.astype(np.float64)
    dd = P.d.astype(np.float64)
    c = (1.0 - beta) * R
    teff = 20  # T_R = ARP / DT
    assert K <= teff and T % K == 0
    bf, c32 = beta.astype(f32), c.astype(f32)
    Bk = np.stack([(beta ** (k + 1)).astype(f32) for k in range(K)], 1)   # rounded powers
    Ph = np.stack([(p ** k).astype(f32) for k in range(K)], 1)
    btab = np.stack([f32(1.0) / (beta ** max(r, 1)).astype(f32) for r in range(K)], 1)
    BK, pK = beta ** K, p ** K
    omb = 1.0 - BK
    ks = np.arange(K)[None, :]
    Vd = np.zeros(rows)   # kernel: carried membrane (double-single, here FP64)
    aw = np.zeros(rows)   # kernel: carried adaptation
    Vx = np.zeros(rows)   # FP64 model
    ax = np.zeros(rows)
    rel = np.zeros(rows, dtype=np.int64)
    mxr = np.zeros(rows)
    worst_near = worst_all = 0.0
    spikes = 0
    for tb in range(0, T, K):
        x = I[:, tb:tb + K]
        cx = _mul(c32[:, None], x)
        L = np.empty((rows, K), f32)
        L[:, 0] = cx[:, 0]
        for k in range(1, K):
            L[:, k] = _fma(bf, L[:, k - 1], cx[:, k])
        vin = np.where(rel > 0, 0.0, Vd).astype(f32)
        part = np.where((rel > 0) & (rel < K))[0]
        vin[part] = _mul(-L[part, rel[part] - 1], btab[part, rel[part]])
        dA = _mul(dd.astype(f32), aw.astype(f32))
        Z = _fma(-dA[:, None], Ph, _fma(Bk, vin[:, None], L)).astype(np.float64)
        mx = np.abs(x).max(1).astype(np.float64)
        mxr = np.maximum(mxr, mx)
        M = np.maximum(np.where(rel > 0, 0.0, np.abs(vin)), R * mx)
        G = (1 + 2.0 ** -6) * (U * (4 * M + 5 * np.abs(dA) + th0) + (4 * K + 4) * U * R * omb * mx
                               + (2 * K + 4) * U * R * mxr)
        Vs = np.where(rel > 0, 0.0, Vx)
        Zs = np.empty((rows, K))
        for k in range(K):
            Vs = beta * Vs + np.where(k >= rel, c * x[:, k], 0.0)
            Zs[:, k] = Vs - dd * p ** k * ax
        adm = ks >= rel[:, None]
        ratio = np.where(adm, np.abs(Z - Zs) / G[:, None], 0.0)
        near = adm & (np.abs(Zs - th0[:, None]) < 1e-3)
        worst_all = max(worst_all, float(ratio.max()))
        if near.any():
            worst_near = max(worst_near, float(ratio[near].max()))
        crossed = adm & (Zs > th0[:, None])
        s = crossed.any(1)
        first = np.where(s, crossed.argmax(1), K)
        spikes += int(s.sum())
        # state entering the next Block (Props 3-5)
        vind = np.where(rel > 0, vin.astype(np.float64), Vd)
        Vx_end = np.where(rel > 0, 0.0, Vx)
        for k in range(K):
            Vx_end = beta * Vx_end + np.where(k >= rel, c * x[:, k], 0.0)
        unit = np.where(s, p ** np.maximum(K - 1 - first, 0), 0.0)
        aw = pK * aw + unit
        ax = pK * ax + unit
        reset = s | (rel >= K)
        Vd = np.where(reset, 0.0, BK * vind + L[:, K - 1].astype(np.float64))
        Vx = np.where(reset, 0.0, Vx_end)
        rel = np.where(s, first + teff - K, np.maximum(rel - K, 0))
    return worst_near, worst_all, spikes


@pytest.mark.parametrize("K, scale, tau_mem, d, seed", [
    (16, 1.0, (10.0, 30.0), (0.0, 0.2), 0),     # the bench workload's neurons, 16-step Blocks
    (16, 6.0, (200.0, 2000.0), (0.5, 2.0), 1),  # slow membranes (beta^K near 1), strong adaptation
    (8, 1.3, (10.0, 30.0), (0.0, 0.2), 2),
    (4, 2.5, (2.0, 5.0), (0.0, 0.2), 3),        # fast membranes, strong drive
    (2, 3.0, (1.0, 3.0), (0.0, 0.5), 4),
])
def test_lane_forward_margin_bound(K, scale, tau_mem, d, seed):
    near, every, spikes = _margin_errors(K, rows=128, T=4000, scale=scale, tau_mem=tau_mem, d=d, seed=seed)
    assert spikes > 200
    assert near < 0.5, near
    assert every < 0.5, every
