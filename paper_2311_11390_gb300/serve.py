"""Continuous-batching server for ALIF simulate / fit requests.

Each request is one population of N neurons (batch 1) driven by 512 Poisson
input channels through its own weights (split-BF16 tensor-core projection plus
a bias), simulated for T steps at its own DT (so its own T_R = ARP / DT).  A
"fit" request also compares the produced spike train with a target train
(van Rossum distance, Supplementary "Neural fits") and returns the gradient of
that loss with respect to the neuron parameters.

Scheduling: requests are admitted, in arrival order, as soon as a slot (a CUDA
stream) is free and their device-memory footprint fits the budget.  Every
admitted request advances chunk by chunk (``chunk`` steps, a multiple of 256);
the neuron state stays on the device between chunks (the forward's final state
is the next chunk's initial state), and each chunk's kernels are enqueued on
the request's stream only after its previous chunk finished, so all active
requests' chunks overlap on the GPU while new requests join as others leave.
A fit request runs its forward chunks, the van Rossum forward, then its
backward chunks last-first (gradients carried between chunks).
Results do not depend on what else runs: each request's kernels see only its
own buffers and fixed chunk boundaries.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import alif, synth

NIN = 512


@dataclass
class Request:
    rid: int
    N: int
    T: int
    dt: float
    fit: bool
    arrival: float = 0.0
    seed: int = 0
    raster: np.ndarray | None = None      # uint32 [NIN, ceil(T/32)]
    W: np.ndarray | None = None           # float32 [N, NIN]
    bias: np.ndarray | None = None        # float32 [N]
    params: synth.NeuronParams | None = None
    target: np.ndarray | None = None      # uint32 [N, ceil(T/32)] (fit only)


@dataclass
class Result:
    rid: int
    spikes: np.ndarray                    # uint32 [N, ceil(T/32)]
    loss: np.ndarray | None = None        # [N] squared van Rossum distance per neuron
    grads: np.ndarray | None = None       # [5, N]: tau_mem, tau_adapt, theta0, d, R
    latency: float = 0.0
    start: float = 0.0
    end: float = 0.0


def make_request(rid, N, T, dt, fit, seed, arrival=0.0, arp=2.0) -> Request:
    """Synthetic request: rates U[10, 50] Hz on 512 channels, W ~ N(0, 2/512), bias U[0.8, 1.6],
    tau_mem U[10, 30] ms, tau_adapt U[100, 500] ms, d U[0, 0.2]; fit targets are a Poisson
    train at 20 Hz."""
    rng = np.random.default_rng(seed)
    params = synth.uniform_params(rng, N, (10.0, 30.0), (100.0, 500.0), 1.0, (0.0, 0.2), 1.0)
    W = (rng.standard_normal((N, NIN)) * math.sqrt(2.0 / NIN)).astype(np.float32)
    bias = rng.uniform(0.8, 1.6, N).astype(np.float32)
    rates = rng.uniform(10.0, 50.0, NIN)
    raster = synth.pack_bits(synth.poisson_raster(rng, 1, NIN, T, rates, dt)[0])
    target = synth.pack_bits(synth.poisson_raster(rng, 1, N, T, np.full(N, 20.0), dt)[0]) if fit else None
    return Request(rid, N, T, dt, fit, arrival, seed, raster, W, bias, params, target)


def request_stream(n, seed=0, N_range=(64, 8192), T_range=(1000, 200000), dts=(0.05, 0.1, 1.0), p_fit=0.3,
                   rate_hz=None):
    """Poisson arrivals (rate_hz; None = all at t=0) of simulate/fit requests with N and T
    log-uniform in the given ranges and DT drawn from `dts`."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for k in range(n):
        if rate_hz:
            t += rng.exponential(1.0 / rate_hz)
        N = int(round(math.exp(rng.uniform(math.log(N_range[0]), math.log(N_range[1])))))
        T = int(round(math.exp(rng.uniform(math.log(T_range[0]), math.log(T_range[1])))))
        dt = float(dts[rng.integers(len(dts))])
        out.append((k, N, T, dt, bool(rng.random() < p_fit), int(rng.integers(1 << 30)), t))
    return out


class _Job:
    """Device-side execution of one request as a sequence of chunk steps."""

    def __init__(self, req: Request, dev, stream, chunk, arp, tau_vr, slope):
        self.req, self.dev, self.stream, self.chunk = req, dev, stream, chunk
        self.arp, self.tau_vr, self.slope = arp, tau_vr, slope
        self.event = torch.cuda.Event()
        self.steps = self._program()
        self.done = False
        self.result = None

    def _program(self):
        r, dev, C = self.req, self.dev, self.chunk
        N, T = r.N, r.T
        nw = (T + 31) // 32
        with torch.cuda.stream(self.stream):
            table = torch.from_numpy(alif.prepare(r.params.tau_mem, r.params.tau_adapt, r.params.theta0,
                                                  r.params.d, r.params.R, r.dt, self.arp)).to(dev, non_blocking=True)
            raster = torch.from_numpy(r.raster.view(np.int32)).to(dev, non_blocking=True)
            Wd = torch.from_numpy(r.W).to(dev, non_blocking=True)
            bias = torch.from_numpy(r.bias).to(dev, non_blocking=True)
            Whi, Wlo = alif.split_bf16(Wd)
            spikes = torch.empty((N, nw), dtype=torch.int32, device=dev)
            nck = alif.ckpt_count(T)
            ckpt = torch.empty((N, nck, 3), dtype=torch.int32, device=dev) if r.fit else None
            state = alif.state_tensor(1, N, device=dev)
            Ic = torch.empty((1, N, C), dtype=torch.float32, device=dev)
            sc = torch.empty((1, N, C // 32), dtype=torch.int32, device=dev)
            ckc = torch.empty((1, N, C // 256, 3), dtype=torch.int32, device=dev) if r.fit else None
            nxt = torch.empty_like(state)
        self.event.record(self.stream)
        yield
        nchunk = (T + C - 1) // C
        bounds = [(c * C, min(T, (c + 1) * C)) for c in range(nchunk)]
        # ---- forward chunks
        for c, (t0, t1) in enumerate(bounds):
            L = t1 - t0
            w0, w1 = t0 // 32, (t1 + 31) // 32
            with torch.cuda.stream(self.stream):
                rc = raster[:, w0:w1].contiguous().unsqueeze(0)
                I = Ic[..., :L] if L == C else torch.empty((1, N, L), dtype=torch.float32, device=dev)
                alif.syn_project(rc, Whi, Wlo, bias, Nin=NIN, T=L, out=I)
                s_out = sc[..., : (L + 31) // 32] if L == C else torch.empty((1, N, (L + 31) // 32),
                                                                               dtype=torch.int32, device=dev)
                ck = None
                if r.fit:
                    ck = ckc[:, :, : (L + 255) // 256] if L == C else torch.empty(
                        (1, N, (L + 255) // 256, 3), dtype=torch.int32, device=dev)
                alif.forward_into(I if I.is_contiguous() else I.contiguous(), table, s_out, ckpt=ck, final=nxt,
                                  init=state)
                spikes[:, w0:w1].copy_(s_out[0])
                if r.fit:
                    ckpt[:, t0 // 256: t0 // 256 + ck.shape[2]].copy_(ck[0])
                state.copy_(nxt)
            self.event.record(self.stream)
            yield
        loss = grads = None
        if r.fit:
            with torch.cuda.stream(self.stream):
                tgt = torch.from_numpy(r.target.view(np.int32)).to(dev, non_blocking=True)
                fck = torch.empty((N, nchunk), dtype=torch.float32, device=dev)
                loss_d = torch.empty((N,), dtype=torch.float32, device=dev)
                alif.vanrossum_forward(spikes, tgt, T, r.dt, self.tau_vr, C, fck, loss_d)
                gcar = torch.zeros((N,), dtype=torch.float32, device=dev)
                gfin = None
                gp_sum = torch.zeros((5, N), dtype=torch.float32, device=dev)
                gS = torch.empty((1, N, C), dtype=torch.float32, device=dev)
            self.event.record(self.stream)
            yield
            for c in range(nchunk - 1, -1, -1):
                t0, t1 = bounds[c]
                L = t1 - t0
                w0, w1 = t0 // 32, (t1 + 31) // 32
                with torch.cuda.stream(self.stream):
                    g = gS[..., :L] if L == C else torch.empty((1, N, L), dtype=torch.float32, device=dev)
                    g = g if g.is_contiguous() else torch.empty((1, N, L), dtype=torch.float32, device=dev)
                    alif.vanrossum_backward(spikes, tgt, T, r.dt, self.tau_vr, t0, t1, fck[:, c].contiguous(),
                                            gcar, g[0])
                    rc = raster[:, w0:w1].contiguous().unsqueeze(0)
                    I = torch.empty((1, N, L), dtype=torch.float32, device=dev)
                    alif.syn_project(rc, Whi, Wlo, bias, Nin=NIN, T=L, out=I)
                    s_c = spikes[:, w0:w1].contiguous().unsqueeze(0)
                    ck = ckpt[:, t0 // 256: t0 // 256 + (L + 255) // 256].contiguous().unsqueeze(0)
                    _, ginit, gp = alif.backward(I, table, s_c, g, ckpt=ck, grad_final=gfin, slope=self.slope,
                                                 want_gI=False, want_ginit=True)
                    gp_sum += gp
                    gfin = ginit
                self.event.record(self.stream)
                yield
            loss, grads = loss_d, gp_sum
        with torch.cuda.stream(self.stream):  # results to pinned host memory, no host sync
            host = lambda x: None if x is None else torch.empty(x.shape, dtype=x.dtype).pin_memory()
            self._out = (host(spikes), host(loss), host(grads))
            for h, d in zip(self._out, (spikes, loss, grads)):
                if h is not None:
                    h.copy_(d, non_blocking=True)
        self.event.record(self.stream)
        yield

    def advance(self) -> bool:
        """Enqueue the next chunk if the previous one finished; True when the request is done."""
        if self.done:
            return True
        if not self.event.query():
            return False
        try:
            next(self.steps)
        except StopIteration:
            sp, lo, gr = self._out
            self.result = Result(self.req.rid, sp.numpy().view(np.uint32),
                                 None if lo is None else lo.numpy(), None if gr is None else gr.numpy())
            self.done = True
        return self.done


class Server:
    def __init__(self, device="cuda", mem_budget=16 << 30, max_active=8, chunk=4096, arp=2.0, tau_vr=5.0,
                 slope=25.0):
        assert chunk % 256 == 0
        self.dev = torch.device(device)
        self.mem_budget, self.max_active, self.chunk = mem_budget, max_active, chunk
        self.arp, self.tau_vr, self.slope = arp, tau_vr, slope
        self.streams = [torch.cuda.Stream(self.dev) for _ in range(max_active)]

    def footprint(self, req: Request) -> int:
        """Device bytes a request holds while active (upper bound)."""
        N, T, C = req.N, req.T, self.chunk
        nw = (T + 31) // 32
        b = NIN * nw * 4 * 2 + N * NIN * 4 * 2 + N * 64 + N * 4      # raster (+chunk copy), W + hi/lo, table, bias
        b += N * nw * 4 + N * (C // 32) * 4 + N * C * 4 + 64 * N     # spikes, chunk spikes, chunk current, states
        if req.fit:
            b += N * ((T + 255) // 256) * 12 * 2 + N * nw * 4 + N * C * 4 * 2 + N * 64
        return b

    def run(self, requests, realtime=True, on_done=None):
        """Serve `requests` (sorted by arrival).  Returns (results by rid, stats)."""
        pending = sorted(requests, key=lambda r: r.arrival)
        for r in pending:
            if self.footprint(r) > self.mem_budget:
                raise ValueError(f"request {r.rid} needs {self.footprint(r)} bytes > budget {self.mem_budget}")
        free = list(range(self.max_active))
        active = {}
        used = 0
        results = {}
        t_start = time.perf_counter()
        steps = 0
        while pending or active:
            now = time.perf_counter() - t_start
            while (pending and free and (not realtime or pending[0].arrival <= now)
                   and used + self.footprint(pending[0]) <= self.mem_budget):
                r = pending.pop(0)
                slot = free.pop(0)
                job = _Job(r, self.dev, self.streams[slot], self.chunk, self.arp, self.tau_vr, self.slope)
                job.slot, job.t_admit = slot, now
                used += self.footprint(r)
                active[r.rid] = job
                next(job.steps)  # enqueue the set-up
            progressed = False
            for rid in list(active):
                job = active[rid]
                if job.advance():
                    t_end = time.perf_counter() - t_start
                    res = job.result
                    res.start, res.end = job.req.arrival if realtime else 0.0, t_end
                    res.latency = t_end - res.start
                    results[rid] = res
                    used -= self.footprint(job.req)
                    free.append(job.slot)
                    del active[rid]
                    steps += job.req.N * job.req.T
                    progressed = True
                    if on_done:
                        on_done(res)
            if not progressed:
                time.sleep(0.0002)
        wall = time.perf_counter() - t_start
        lat = np.array([r.latency for r in results.values()])
        stats = {"requests": len(results), "wall_s": wall, "neuron_steps": steps,
                 "neuron_steps_per_s": steps / wall if wall > 0 else None,
                 "p50_s": float(np.percentile(lat, 50)) if len(lat) else None,
                 "p99_s": float(np.percentile(lat, 99)) if len(lat) else None}
        return results, stats
