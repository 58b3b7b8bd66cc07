"""The forward kernels' margin error bounds, checked on the CPU (no GPU).

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

`fwd_kernel` (a warp per row, windows of W = 32 E steps) scans a window with two E/2-step chains
per lane, five shuffle levels over the lane totals and a rebuild pass, and carries the membrane
into the next window in FP32.  Its bound counts at most E + 16 roundings on any term's path:

    G = (1 + 2^-6) u ((E + 17) max(|v_in|, R max_win|I|) + 4 |d a| + theta0
                      + (E + 16) (beta^W / (1 - beta^W) max_row|v_in| + R max_row|I|)),

without the carried terms in a rescan after a spike (it starts from an exact 0).  The second
test restates that scan (the shuffle levels read the lane totals before the level) and checks
the bound over whole windows with their spikes and rescans.
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


def _warp_scan(q, bf, bh, Bl, Bk, E):
    """The warp kernel's decayed scan of q [rows, 32 lanes, E]: per lane two H-step FMA chains
    from zero, the lane total, five shuffle levels (lane l adds Bl[lev] times lane l - 2^lev),
    the membrane entering each lane, then the rebuild with the rounded powers Bk."""
    H = E // 2
    L = np.empty_like(q)
    L[:, :, 0], L[:, :, H] = q[:, :, 0], q[:, :, H]
    for k in range(1, H):
        L[:, :, k] = _fma(bf[:, None], L[:, :, k - 1], q[:, :, k])
        L[:, :, H + k] = _fma(bf[:, None], L[:, :, H + k - 1], q[:, :, H + k])
    tot = _fma(bh[:, None], L[:, :, H - 1], L[:, :, E - 1])
    for lev in range(5):
        dl = 1 << lev
        prev = tot.copy()
        tot[:, dl:] = _fma(Bl[:, lev][:, None], prev[:, :-dl], prev[:, dl:])
    P = np.zeros_like(tot)
    P[:, 1:] = tot[:, :-1]
    V = np.empty_like(q)
    for k in range(H):
        V[:, :, k] = _fma(Bk[:, k][:, None], P, L[:, :, k])
    for k in range(H):
        V[:, :, H + k] = _fma(Bk[:, k][:, None], V[:, :, H - 1], L[:, :, H + k])
    return V


def _warp_margin_errors(E, I, P, dt, arp):
    """Largest |Z - Z*| / G over admitted margins near threshold and over all of them, spikes."""
    rows, T = I.shape
    W = 32 * E
    H = E // 2
    beta = np.exp(-dt / P.tau_mem.astype(np.float64))
    p = np.exp(-dt / P.tau_adapt.astype(np.float64))
    R, th0, d = P.R.astype(np.float64), P.theta0.astype(np.float64), P.d.astype(np.float64)
    c = (1.0 - beta) * R
    teff = max(int(round(arp / dt)), 2)
    bf, c32 = beta.astype(f32), c.astype(f32)
    Bk = np.stack([(beta ** (k + 1)).astype(f32) for k in range(H)], 1)
    bh = (beta ** H).astype(f32)
    Bl = np.stack([(beta ** (E << lev)).astype(f32) for lev in range(5)], 1)
    bW = beta ** W
    us = U * (1 + 2.0 ** -6)
    gC = (E + 16) * us * np.minimum(bW / np.maximum(1.0 - bW, 2.0 ** -20), 2.0 ** 20)
    gM, gD, gR, g0 = (E + 17) * us, 4 * us, (E + 16) * us * R, us * th0
    ptab = np.stack([p ** j for j in range(W + 1)], 1)
    ptab32 = ptab.astype(f32)
    t = np.arange(W)
    ri = np.arange(rows)
    Vin = np.zeros(rows, f32)
    Vx = np.zeros(rows)
    aw = np.zeros(rows)
    ax = np.zeros(rows)
    rel = np.zeros(rows, dtype=np.int64)
    vmr = np.zeros(rows)
    mxr = np.zeros(rows)
    worst_near = worst_all = 0.0
    spikes = 0
    for wi in range(T // W):
        x = I[:, wi * W:(wi + 1) * W]
        mx = np.abs(x).max(1).astype(np.float64)
        mxr = np.maximum(mxr, mx)
        vmr = np.maximum(vmr, np.abs(Vin.astype(np.float64)))
        cx = _mul(c32[:, None], x)
        start = np.clip(rel, 0, W)
        first = np.ones(rows, bool)     # the round that carries the entering membrane
        t1 = np.zeros(rows, dtype=np.int64)  # a[t] = A p^(t - t1)
        A, Ax = aw.copy(), ax.copy()
        active = np.ones(rows, bool)
        endV, endVx = np.zeros(rows, f32), np.zeros(rows)
        spk = np.zeros(rows, bool)
        s2_last = np.zeros(rows, dtype=np.int64)
        while active.any():
            q = np.where(t[None, :] >= start[:, None], cx, f32(0)).reshape(rows, 32, E).copy()
            q[:, 0, 0] = np.where(first, _fma(bf, Vin, q[:, 0, 0]), q[:, 0, 0])
            V = _warp_scan(q, bf, bh, Bl, Bk, E).reshape(rows, W)
            xin = np.where(t[None, :] >= start[:, None], c[:, None] * x, 0.0)
            Vs = np.where(first, Vx, 0.0)
            Vex = np.empty((rows, W))
            for k in range(W):
                Vs = beta * Vs + xin[:, k]
                Vex[:, k] = Vs
            pidx = np.maximum(t[None, :] - t1[:, None], 0)
            dA = _mul(d.astype(f32), A.astype(f32))
            Z = _fma(-dA[:, None], np.take_along_axis(ptab32, pidx, 1), V).astype(np.float64)
            Zx = Vex - d[:, None] * Ax[:, None] * np.take_along_axis(ptab, pidx, 1)
            M = np.where(first, np.maximum(np.abs(Vin.astype(np.float64)), R * mx), R * mx)
            G = gM * M + gD * np.abs(dA) + g0 + np.where(first, gC * vmr + gR * mxr, 0.0)
            adm = (t[None, :] >= start[:, None]) & active[:, None]
            ratio = np.where(adm, np.abs(Z - Zx) / G[:, None], 0.0)
            worst_all = max(worst_all, float(ratio.max()))
            near = adm & (np.abs(Zx - th0[:, None]) < 1e-3)
            if near.any():
                worst_near = max(worst_near, float(ratio[near].max()))
            cross = adm & (Zx > th0[:, None])
            has = cross.any(1)
            tau = np.where(has, cross.argmax(1), W)
            done = active & ~has
            endV, endVx = np.where(done, V[:, W - 1], endV), np.where(done, Vex[:, W - 1], endVx)
            sp = active & has
            spikes += int(sp.sum())
            decay = ptab[ri, np.clip(tau - t1, 0, W)]
            A = np.where(sp, p * A * decay + 1.0, A)        # a[tau + 1] (Eq 5)
            Ax = np.where(sp, p * Ax * decay + 1.0, Ax)
            t1 = np.where(sp, tau + 1, t1)
            s2 = tau + teff
            spk |= sp
            s2_last = np.where(sp, s2, s2_last)
            out = sp & (s2 >= W)
            endV, endVx = np.where(out, f32(0), endV), np.where(out, 0.0, endVx)
            start = np.where(sp, s2, start)
            first &= ~sp
            active = sp & (s2 < W)
        Vin, Vx = endV.astype(f32), endVx
        aw = np.where(spk, A * ptab[ri, np.clip(W - t1, 0, W)], aw * ptab[:, W])
        ax = np.where(spk, Ax * ptab[ri, np.clip(W - t1, 0, W)], ax * ptab[:, W])
        rel = np.where(spk, s2_last - W, rel - W)
    return worst_near, worst_all, spikes


@pytest.mark.parametrize("E, workload, scale, tau_mem, seed", [
    (16, "fit", 1.0, None, 0),               # the neuron fit's OU current, 512-step windows
    (8, "ff", 1.0, (10.0, 30.0), 0),         # the bench workload's neurons, 256-step windows
    (8, "ff", 3.0, (200.0, 2000.0), 1),      # slow membranes: the FP32 carry's errors persist
    (8, "ff", 3.0, (1.0, 3.0), 2),           # fast membranes, strong drive
    (16, "ff", 1.5, (10.0, 30.0), 3),
])
def test_warp_forward_margin_bound(E, workload, scale, tau_mem, seed):
    if workload == "fit":
        w = synth.neuron_fit(seed=seed, N=128, T=512 * 60)
        I = (w.I[0] * scale).astype(f32)
    else:
        w = synth.feedforward(seed=seed, B=1, Nin=1000, N=128, T=32 * E * 16, dt=0.1, arp=2.0, tau_mem=tau_mem)
        I = (project.project(w.W, w.S_in, w.bias)[0] * scale).astype(f32)
    near, every, spikes = _warp_margin_errors(E, I, w.params, w.dt, w.arp)
    assert spikes > 100
    assert near < 0.5, near
    assert every < 0.5, every
