"""Continuous-batching server for ALIF simulate / fit requests.

Each request is one population of N neurons (batch 1) driven by 512 Poisson
input channels through its own weights (split-BF16 tensor-core projection plus
a bias), simulated for T steps at its own DT (so its own T_R = ARP / DT).  A
"fit" request also compares the produced spike train with a target train
(van Rossum distance, Supplementary "Neural fits") and returns the gradient of
that loss with respect to the neuron parameters.

Device layout: every admitted request owns a contiguous range of rows in one
row arena, allocated once with the server: its prepared neuron constants (the
table carries each row's own T_R, so requests of different DT share a launch),
its state entering the next chunk (two buffers, swapped every round), and the
round's current, spike and checkpoint chunks.  Per-slot chunk buffers for the
backward of fit requests are allocated once as well; nothing is allocated per
chunk.

Scheduling: requests are admitted in arrival order when a slot is free, a row
range fits and their device-memory footprint fits the budget.  Every round
advances all requests in their forward phase by one chunk: each request's
projection writes its rows of the round's current, then ONE block-forward
launch covers the row range of all of them (rows are independent, so each
request's result does not depend on its neighbours; rows of requests in their
backward phase and free rows inside the range are simulated too and ignored).
Rounds are enqueued on one compute stream, at most two ahead of the GPU.  A
fit request that finishes its forward enqueues its whole backward (van Rossum
loss, then its backward chunks last-first) on its slot's stream at once, where
it overlaps the following rounds.  Inputs (raster, weights, bias, fit target)
are generated on the device from the request's seed at admission.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass

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


@dataclass
class Result:
    rid: int
    spikes: np.ndarray                    # uint32 [N, ceil(T/32)] (bits at t >= T zero)
    loss: np.ndarray | None = None        # [N] squared van Rossum distance per neuron
    grads: np.ndarray | None = None       # [5, N]: tau_mem, tau_adapt, theta0, d, R
    latency: float = 0.0
    start: float = 0.0
    end: float = 0.0


def make_request(rid, N, T, dt, fit, seed, arrival=0.0) -> Request:
    return Request(rid, N, T, dt, fit, arrival, seed)


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


def request_params(req: Request) -> synth.NeuronParams:
    """tau_mem U[10, 30] ms, tau_adapt U[100, 500] ms, theta0 1, d U[0, 0.2], R 1 (host, seeded)."""
    rng = np.random.default_rng(req.seed)
    return synth.uniform_params(rng, req.N, (10.0, 30.0), (100.0, 500.0), 1.0, (0.0, 0.2), 1.0)


def materialize(req: Request, device, chunk=16384):
    """The request's inputs on the device, generated from its seed: rates U[10, 50] Hz on 512
    channels -> raster [NIN, ceil(T/32)] words; W ~ N(0, 2/512) [N, NIN]; bias U[0.8, 1.6];
    fit target: a 20 Hz Poisson train [N, ceil(T/32)] words."""
    g = torch.Generator(device=device).manual_seed(req.seed)
    W = torch.randn((req.N, NIN), generator=g, device=device) * math.sqrt(2.0 / NIN)
    bias = 0.8 + 0.8 * torch.rand((req.N,), generator=g, device=device)
    rates = 10.0 + 40.0 * torch.rand((NIN, 1), generator=g, device=device)
    nw = (req.T + 31) // 32
    raster = torch.zeros((NIN, nw), dtype=torch.int32, device=device)
    target = torch.zeros((req.N, nw), dtype=torch.int32, device=device) if req.fit else None
    for t0 in range(0, req.T, chunk):  # bounded temporaries: one chunk of 0/1 floats at a time
        L = min(chunk, req.T - t0)
        S = (torch.rand((NIN, L), generator=g, device=device) < rates * (req.dt * 1e-3)).to(torch.float32)
        raster[:, t0 // 32: t0 // 32 + (L + 31) // 32] = alif.pack_spikes(S)
        if req.fit:
            Y = (torch.rand((req.N, L), generator=g, device=device) < 20.0 * req.dt * 1e-3).to(torch.float32)
            target[:, t0 // 32: t0 // 32 + (L + 31) // 32] = alif.pack_spikes(Y)
    return raster, W, bias, target


class _Rows:
    """First-fit allocator of contiguous row ranges in the arena."""

    def __init__(self, n):
        self.free = [(0, n)]

    def alloc(self, k):
        for i, (a, b) in enumerate(self.free):
            if b - a >= k:
                self.free[i] = (a + k, b)
                if a + k == b:
                    del self.free[i]
                return a
        return None

    def release(self, a, k):
        self.free.append((a, a + k))
        self.free.sort()
        merged = []
        for x, y in self.free:
            if merged and merged[-1][1] == x:
                merged[-1] = (merged[-1][0], y)
            else:
                merged.append((x, y))
        self.free = merged


class _Job:
    def __init__(self, req, row0, slot, table_host):
        self.req, self.row0, self.slot = req, row0, slot
        self.table_host = table_host
        self.nchunk = 0
        self.next_chunk = 0
        self.done_event = None
        self.out = None
        self.t_admit = 0.0


class Server:
    def __init__(self, device="cuda", mem_budget=16 << 30, max_active=8, chunk=4096, arp=2.0, tau_vr=5.0,
                 slope=25.0, rows_max=None, n_max=8192):
        assert chunk % 256 == 0
        self.dev = torch.device(device)
        self.mem_budget, self.max_active, self.chunk = mem_budget, max_active, chunk
        self.arp, self.tau_vr, self.slope, self.n_max = arp, tau_vr, slope, n_max
        self.rows_max = rows_max or max_active * n_max
        R, C, dev = self.rows_max, chunk, self.dev
        self.table = torch.zeros((R, alif.NEURON_FLOATS), dtype=torch.float32, device=dev)
        self.state = [torch.zeros((1, R, 3), dtype=torch.int32, device=dev) for _ in range(2)]
        self.I = torch.zeros((1, R, C), dtype=torch.float32, device=dev)
        self.spk = torch.zeros((1, R, C // 32), dtype=torch.int32, device=dev)
        self.ckc = torch.zeros((1, R, C // 256, 3), dtype=torch.int32, device=dev)
        self.compute = torch.cuda.Stream(dev)
        self.streams = [torch.cuda.Stream(dev) for _ in range(max_active)]
        # per-slot buffers (one chunk of current and of dL/dS), flat so that any [1, N, L] view of
        # their start is contiguous
        self.slot_I = [torch.empty(n_max * C, dtype=torch.float32, device=dev) for _ in range(max_active)]
        self.slot_g = [torch.empty(n_max * C, dtype=torch.float32, device=dev) for _ in range(max_active)]

    def _slot_view(self, buf, N, L):
        return buf[: N * L].view(1, N, L)

    def footprint(self, req: Request) -> int:
        """Device bytes a request holds while active, beyond the arenas (upper bound)."""
        N, T = req.N, req.T
        nw = (T + 31) // 32
        b = NIN * nw * 4 + N * NIN * 4 * 3 + N * 4 + N * nw * 4    # raster, W (+ hi/lo), bias, spikes
        if req.fit:
            b += N * nw * 4 + N * ((T + 255) // 256) * 12 + N * 64 * 4  # target, checkpoints, loss state
        return b

    # ------------------------------------------------------------ request life
    def _admit(self, req, slot, row0):
        dev, C = self.dev, self.chunk
        p = request_params(req)
        job = _Job(req, row0, slot, alif.prepare(p.tau_mem, p.tau_adapt, p.theta0, p.d, p.R, req.dt, self.arp))
        N, T = req.N, req.T
        with torch.cuda.stream(self.compute):
            job.raster, W, job.bias, job.target = materialize(req, dev)
            job.W = W
            job.Whi, job.Wlo = alif.split_bf16(W)
            job.spikes = torch.zeros((N, (T + 31) // 32), dtype=torch.int32, device=dev)
            job.ckpt = torch.empty((N, alif.ckpt_count(T), 3), dtype=torch.int32, device=dev) if req.fit else None
            self.table[row0:row0 + N].copy_(torch.from_numpy(job.table_host), non_blocking=True)
            for s in self.state:
                s[:, row0:row0 + N].zero_()  # rest state entering step 0
        job.nchunk = (T + C - 1) // C
        return job

    def _project(self, job, c):
        """Current of chunk c of `job` into its arena rows (zero beyond the request's T)."""
        C, r = self.chunk, job.req
        t0 = c * C
        L = min(C, r.T - t0)
        rows = slice(job.row0, job.row0 + r.N)
        Ic = self.I[:, rows, :]
        rc = job.raster[:, t0 // 32: t0 // 32 + (L + 31) // 32].contiguous().unsqueeze(0)
        if L == C:
            alif.syn_project(rc, job.Whi, job.Wlo, job.bias, Nin=NIN, T=C, out=Ic)
        else:
            tmp = self._slot_view(self.slot_I[job.slot], r.N, L)
            alif.syn_project(rc, job.Whi, job.Wlo, job.bias, Nin=NIN, T=L, out=tmp)
            Ic[..., :L].copy_(tmp)
            Ic[..., L:].zero_()

    def _collect(self, job, c):
        """Chunk c's spikes (and checkpoints) from the arena into the request's buffers."""
        C, r = self.chunk, job.req
        t0 = c * C
        L = min(C, r.T - t0)
        rows = slice(job.row0, job.row0 + r.N)
        w0, nwc = t0 // 32, (L + 31) // 32
        job.spikes[:, w0:w0 + nwc].copy_(self.spk[0, rows, :nwc])
        if L % 32:
            job.spikes[:, w0 + nwc - 1] &= (1 << (L % 32)) - 1
        if r.fit:
            k0, nk = t0 // 256, (L + 255) // 256
            job.ckpt[:, k0:k0 + nk].copy_(self.ckc[0, rows, :nk])

    def _fit_backward(self, job):
        """Van Rossum loss and the parameter gradients, enqueued at once on the slot's stream."""
        r, C, dev = job.req, self.chunk, self.dev
        N, T = r.N, r.T
        st = self.streams[job.slot]
        fwd_done = torch.cuda.Event()
        fwd_done.record(self.compute)
        st.wait_event(fwd_done)
        with torch.cuda.stream(st):
            fck = torch.empty((N, job.nchunk), dtype=torch.float32, device=dev)
            loss = torch.empty((N,), dtype=torch.float32, device=dev)
            alif.vanrossum_forward(job.spikes, job.target, T, r.dt, self.tau_vr, C, fck, loss)
            gcar = torch.zeros((N,), dtype=torch.float32, device=dev)
            gp_sum = torch.zeros((5, N), dtype=torch.float32, device=dev)
            gp = torch.empty((5, N), dtype=torch.float32, device=dev)
            ginit = torch.empty((1, N, 2), dtype=torch.float32, device=dev)
            gfin = torch.empty((1, N, 2), dtype=torch.float32, device=dev)
            table = torch.from_numpy(job.table_host).to(dev, non_blocking=True)
            ws = torch.empty(alif.workspace_size(1, N), dtype=torch.uint8, device=dev)
            have_fin = False
            for c in range(job.nchunk - 1, -1, -1):
                t0 = c * C
                L = min(C, T - t0)
                g = self._slot_view(self.slot_g[job.slot], N, L)
                I = self._slot_view(self.slot_I[job.slot], N, L)
                alif.vanrossum_backward(job.spikes, job.target, T, r.dt, self.tau_vr, t0, t0 + L,
                                        fck[:, c].contiguous(), gcar, g[0])
                rc = job.raster[:, t0 // 32: t0 // 32 + (L + 31) // 32].contiguous().unsqueeze(0)
                alif.syn_project(rc, job.Whi, job.Wlo, job.bias, Nin=NIN, T=L, out=I)
                s_c = job.spikes[:, t0 // 32: t0 // 32 + (L + 31) // 32].contiguous().unsqueeze(0)
                ck = job.ckpt[:, t0 // 256: t0 // 256 + (L + 255) // 256].contiguous().unsqueeze(0)
                alif.backward(I, table, s_c, g, ckpt=ck, grad_final=gfin if have_fin else None, slope=self.slope,
                              want_gI=False, want_ginit=True, workspace=ws, out_gp=gp, out_ginit=ginit)
                gp_sum += gp
                gfin.copy_(ginit)
                have_fin = True
        job.loss, job.grads = loss, gp_sum
        return st

    def _finish(self, job, stream):
        """Results to pinned host memory on `stream`; completion event recorded there."""
        with torch.cuda.stream(stream):
            host = lambda x: None if x is None else torch.empty(x.shape, dtype=x.dtype).pin_memory()
            outs = (job.spikes, getattr(job, "loss", None), getattr(job, "grads", None))
            job.out = tuple(host(x) for x in outs)
            for h, d in zip(job.out, outs):
                if h is not None:
                    h.copy_(d, non_blocking=True)
            job.done_event = torch.cuda.Event()
            job.done_event.record(stream)

    # ----------------------------------------------------------------- the loop
    def run(self, requests, realtime=True, on_done=None):
        """Serve `requests` (sorted by arrival).  Returns (results by rid, stats)."""
        pending = sorted(requests, key=lambda r: r.arrival)
        for r in pending:
            if self.footprint(r) > self.mem_budget:
                raise ValueError(f"request {r.rid} needs {self.footprint(r)} bytes > budget {self.mem_budget}")
            if r.N > self.n_max or r.N > self.rows_max:
                raise ValueError(f"request {r.rid}: N = {r.N} exceeds the server's {self.n_max} rows per request")
        rows = _Rows(self.rows_max)
        free = list(range(self.max_active))
        forward, finishing = [], []
        used = 0
        results, steps = {}, 0
        rounds = []  # completion events of enqueued rounds
        cur = 0      # state buffer holding the state entering the next round
        t_start = time.perf_counter()
        while pending or forward or finishing:
            now = time.perf_counter() - t_start
            # ---- admission
            while pending and free and (not realtime or pending[0].arrival <= now) \
                    and used + self.footprint(pending[0]) <= self.mem_budget:
                row0 = rows.alloc(pending[0].N)
                if row0 is None:
                    break
                r = pending.pop(0)
                job = self._admit(r, free.pop(0), row0)
                job.t_admit = now
                used += self.footprint(r)
                forward.append(job)
            # ---- one round: every forward-phase request advances one chunk, one forward launch
            if forward:
                if len(rounds) >= 2:  # at most two rounds ahead of the GPU
                    rounds.pop(0).synchronize()
                with torch.cuda.stream(self.compute):
                    for job in forward:
                        self._project(job, job.next_chunk)
                    lo = min(j.row0 for j in forward)
                    hi = max(j.row0 + j.req.N for j in forward)
                    sl = slice(lo, hi)
                    alif.forward_into(self.I[:, sl], self.table[sl], self.spk[:, sl], ckpt=self.ckc[:, sl],
                                      final=self.state[1 - cur][:, sl], init=self.state[cur][:, sl])
                    for job in forward:
                        self._collect(job, job.next_chunk)
                        job.next_chunk += 1
                    ev = torch.cuda.Event()
                    ev.record(self.compute)
                    rounds.append(ev)
                cur = 1 - cur
                still = []
                for job in forward:
                    if job.next_chunk < job.nchunk:
                        still.append(job)
                    else:
                        if job.req.fit:
                            st = self._fit_backward(job)
                        else:
                            st = self.compute
                        self._finish(job, st)
                        finishing.append(job)
                forward = still
            # ---- completions
            progressed = False
            for job in list(finishing):
                if job.done_event.query():
                    t_end = time.perf_counter() - t_start
                    sp, lo_, gr = job.out
                    res = Result(job.req.rid, sp.numpy().view(np.uint32), None if lo_ is None else lo_.numpy(),
                                 None if gr is None else gr.numpy())
                    res.start = job.req.arrival if realtime else 0.0
                    res.end = t_end
                    res.latency = t_end - res.start
                    results[job.req.rid] = res
                    used -= self.footprint(job.req)
                    rows.release(job.row0, job.req.N)
                    free.append(job.slot)
                    finishing.remove(job)
                    steps += job.req.N * job.req.T
                    progressed = True
                    if on_done:
                        on_done(res)
            if not forward and not progressed:
                if finishing or (pending and realtime):
                    time.sleep(0.0002)
        torch.cuda.synchronize(self.dev)
        wall = time.perf_counter() - t_start
        lat = np.array([r.latency for r in results.values()])
        stats = {"requests": len(results), "wall_s": wall, "neuron_steps": steps,
                 "neuron_steps_per_s": steps / wall if wall > 0 else None,
                 "p50_s": float(np.percentile(lat, 50)) if len(lat) else None,
                 "p99_s": float(np.percentile(lat, 99)) if len(lat) else None}
        return results, stats
