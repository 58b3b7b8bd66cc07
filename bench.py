#!/usr/bin/env python
"""Benchmark of the ARP-blocked ALIF hot path on GB300 -- prints ONE JSON line.

Workload (default): the feedforward ALIF layer -- 1000 Poisson input channels
(rates U[10, 50] Hz) through dense N(0, 2/1000) weights plus a per-neuron bias
U[0.8, 1.6] into N = 1024 ALIF neurons, batch 32, T = 16000 steps at DT = 0.1 ms,
ARP = 2 ms (T_R = 20); tau_mem U[10, 30] ms, tau_adapt U[100, 500] ms, d U[0, 0.2].
Synthetic, seeded inputs (the paper's speed benchmark also uses synthetic
Poisson spikes).  One step = the whole hot path:
    synaptic projection (split-BF16 tcgen05 GEMM over the spike raster)
    -> block forward (spikes + block-boundary states)
    -> block backward (surrogate gradient; dL/dI and parameter gradients)
with a fixed synthetic upstream gradient dL/dS resident on the device.

--impl reference times the FP64 CPU oracle (the plain step-by-step model) on
the host cores over a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = dict(B=32, Nin=1000, N=1024, T=16000, dt=0.1, arp=2.0)
METRIC = "ALIF neuron-steps/s, fwd+bwd (projection + block forward + block backward)"
UNIT = "neuron-steps/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--T", type=int, default=WORKLOAD["T"])
    ap.add_argument("--B", type=int, default=WORKLOAD["B"])
    ap.add_argument("--arp", type=float, default=WORKLOAD["arp"])
    ap.add_argument("--no-seq", action="store_true", help="skip the sequential-kernel comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-fit", action="store_true", help="skip the neuron-fit configuration")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving stream")
    ap.add_argument("--no-train", action="store_true", help="skip the classification training step")
    ap.add_argument("--no-sweep", action="store_true", help="skip the T x ARP sweep and the small population")
    ap.add_argument("--no-rec", action="store_true", help="skip the recurrent-layer line")
    ap.add_argument("--serve-requests", type=int, default=1000)
    ap.add_argument("--train-T", type=int, nargs="*", default=[1000, 10000],
                    help="sequence lengths of the classification training line (1000: DT 1 ms, 10000: DT 0.1 ms)")
    return ap.parse_args()


# ------------------------------------------------------------ distributed
def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def max_over_ranks(x: float, world: int, device=None) -> float:
    """Max of a per-rank float over all ranks (identity when world == 1)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower() in ("active", "1", "yes"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------- inputs
def make_inputs(seed: int, B: int, T: int, arp: float):
    from paper_2311_11390_gb300 import synth
    w = synth.feedforward(seed=seed, B=B, Nin=WORKLOAD["Nin"], N=WORKLOAD["N"], T=T, dt=WORKLOAD["dt"], arp=arp)
    return w, synth.pack_bits(w.S_in)


def source_hash(files) -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2311_11390_gb300", "csrc")
    for fn in files:
        h.update(open(os.path.join(csrc, fn), "rb").read())
    return h.hexdigest()


def profiled_traffic(kernel: str, units: int):
    """DRAM bytes per launch from the committed ncu summary (bytes per neuron-step of a
    smaller capture, scaled to `units` neuron-steps), or None if the kernel's source
    changed since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        data = json.load(open(path))
    except (OSError, ValueError):
        return None
    ent = data.get(kernel)
    if not ent or ent.get("source_sha256") != source_hash(ent.get("kernel_sources", [])):
        return None
    return ent["bytes_per_neuron_step"] * units


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ------------------------------------------------------------- CPU oracle
def cpu_oracle_sample(w, rows: int, nthreads: int):
    """Oracle (projection in float64 + step-by-step forward + BPTT) on batch element 0,
    neurons [0, rows), full T.  Returns (neuron_steps, seconds)."""
    from oracle import project, ref
    Wsub = w.W[:rows]
    t0 = time.perf_counter()
    I = project.project(Wsub, w.S_in[:1], w.bias[:rows]).astype(np.float32)
    P = ref.Params(*(np.asarray(getattr(w.params, k)[:rows], np.float64)
                     for k in ("tau_mem", "tau_adapt", "theta0", "d", "R")))
    rng = np.random.default_rng(1)
    gS = rng.standard_normal(I.shape)
    ref.forward(I, P, w.dt, w.arp, nthreads=nthreads, records=False)
    ref.backward(I, P, w.dt, w.arp, gS, nthreads=nthreads)
    return rows * I.shape[-1], time.perf_counter() - t0


def run_reference(args, rank, world):
    """Reference arm: the FP64 oracle on the host cores, bounded sample per step."""
    if rank != 0:
        return
    from oracle import ref
    ref.build()
    cores = os.cpu_count() or 1
    w, _ = make_inputs(0, 1, args.T, args.arp)
    rows = 128
    for _ in range(args.warmup):
        cpu_oracle_sample(w, rows, cores)
    tot_steps, tot_s = 0, 0.0
    for _ in range(args.steps):
        n, s = cpu_oracle_sample(w, rows, cores)
        tot_steps += n
        tot_s += s
    value = tot_steps / tot_s
    sample = f"batch element 0, neurons 0..{rows - 1}, full T={args.T} per step (projection+fwd+bwd)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "feedforward ALIF layer, B=%d Nin=1000 N=1024 T=%d DT=0.1ms ARP=%gms"
                       % (args.B, args.T, args.arp), "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------- extra configurations
def fit_config(dev, with_seq=True):
    """Neuron fitting at fine DT: 1024 candidate parameter sets, one shared OU current, T = 400000
    at DT = 0.05 ms (T_R = 40); forward + backward with grad_I = NULL (parameter gradients only),
    blocked vs the plain sequential kernels on the same inputs."""
    import torch
    from paper_2311_11390_gb300 import alif, synth
    w = synth.neuron_fit(seed=0, N=1024, T=400000)
    I = torch.from_numpy(w.I).to(dev)
    N, T = 1024, 400000
    table = alif.neuron_table(w.params.tau_mem, w.params.tau_adapt, w.params.theta0, w.params.d, w.params.R,
                              w.dt, w.arp, device=dev)
    g = torch.Generator(device=dev).manual_seed(7)
    gS = torch.randn((1, N, T), device=dev, generator=g)
    spikes = torch.empty((1, N, (T + 31) // 32), dtype=torch.int32, device=dev)
    ckpt = torch.empty((1, N, alif.ckpt_count(T), 3), dtype=torch.int32, device=dev)
    ws = torch.empty(alif.workspace_size(1, N), dtype=torch.uint8, device=dev)
    gp = torch.empty((5, N), device=dev)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b) / reps

    f_ms = timed(lambda: alif.forward_into(I, table, spikes, ckpt=ckpt), 5)
    b_ms = timed(lambda: alif.backward(I, table, spikes, gS, ckpt=ckpt, workspace=ws, want_gI=False, out_gp=gp), 5)
    out = {"workload": "neuron fit: B=1, N=1024 candidates, T=400000, DT=0.05 ms, ARP=2 ms (T_R=40), OU current",
           "fwd_ms": f_ms, "bwd_ms": b_ms, "fwd_value": N * T / (f_ms / 1e3),
           "fwd_bwd_value": N * T / ((f_ms + b_ms) / 1e3)}
    if with_seq:
        vtr, atr = torch.empty_like(I), torch.empty_like(I)
        sf = timed(lambda: alif.forward_into(I, table, spikes, v=vtr, a=atr, seq=True), 1)
        sb = timed(lambda: alif.backward(I, table, spikes, gS, v_trace=vtr, a_trace=atr, seq=True, workspace=ws,
                                         want_gI=False, out_gp=gp), 1)
        stg = timed(lambda: alif.forward_into(I, table, spikes, seq="staged"), 1)
        out.update({"seq_fwd_ms": sf, "seq_bwd_ms": sb, "staged_seq_fwd_ms": stg,
                    "blocked_over_sequential_fwd": sf / f_ms, "blocked_over_staged_fwd": stg / f_ms,
                    "blocked_over_sequential_fwd_bwd": (sf + sb) / (f_ms + b_ms)})
    return out


def serve_config(dev, n_req):
    """Serving stream: simulate/fit requests with N log-uniform [64, 8192], T log-uniform
    [1e3, 2e5], DT in {0.05, 0.1, 1} ms, 30% fits.  After a short untimed warm-up, capacity is
    measured with every request present at t = 0; then the same requests arrive as a Poisson
    stream at 70% of it."""
    from paper_2311_11390_gb300 import serve
    specs = serve.request_stream(n_req, seed=5)
    reqs = [serve.make_request(rid, N, T, dt, fit, sd) for rid, N, T, dt, fit, sd, _ in specs]
    srv = serve.Server(device=dev, mem_budget=64 << 30, max_active=8, chunk=16384)
    srv.run(reqs[:40], realtime=False)  # warm-up: first launches of every shape, allocator growth
    _, sat = srv.run(reqs, realtime=False)
    cap = sat["requests"] / sat["wall_s"]
    rng = np.random.default_rng(6)
    t = 0.0
    for r in reqs:
        t += rng.exponential(1.0 / (0.7 * cap))
        r.arrival = t
    _, st = srv.run(reqs, realtime=True)
    return {"workload": f"{n_req} requests, N log-U[64,8192], T log-U[1e3,2e5], DT in {{0.05,0.1,1}} ms, 30% fit",
            "requests": st["requests"], "capacity_req_per_s": cap, "arrival_rate_req_per_s": 0.7 * cap,
            "p50_ms": 1e3 * st["p50_s"], "p99_ms": 1e3 * st["p99_s"], "neuron_steps_per_s": st["neuron_steps_per_s"],
            "saturated_neuron_steps_per_s": sat["neuron_steps_per_s"], "wall_s": st["wall_s"],
            "engine": "row arena, one forward launch per chunk round over all requests in their forward phase, "
                      "fit backward enqueued at once per request on its slot stream"}


def train_config(dev, steps=3, Ts=(1000, 10000)):
    """Classification training step (forward + backward through torch.autograd): 700 Poisson
    input channels with class-dependent rate profiles (20 classes) -> 256 ALIF -> 256 ALIF ->
    20-class leaky readout, cross-entropy, batch 128, at (T=1000, DT=1 ms) and (T=10000,
    DT=0.1 ms), ARP 2 ms.  Inputs are drawn on the device from a seeded generator with the
    same rate profiles; weights use the classification initialisation."""
    import torch
    from paper_2311_11390_gb300 import alif, network
    out = {}
    B, C_in, H, K = 128, 700, (256, 256), 20
    for T, dt in ((T, 1.0 if T == 1000 else 0.1) for T in Ts if T in (1000, 10000)):
        g = torch.Generator(device=dev).manual_seed(11)
        labels = torch.randint(0, K, (B,), generator=g, device=dev, dtype=torch.int64)
        j = torch.arange(C_in, device=dev, dtype=torch.float32)
        mu = 35.0 * labels.to(torch.float32) + 17.0
        rates = 5.0 + 45.0 * torch.exp(-((j[None, :] - mu[:, None]) ** 2) / (2 * 50.0 ** 2))
        prob = (rates * dt * 1e-3)[:, :, None]
        words = torch.empty((B, C_in, (T + 31) // 32), dtype=torch.int32, device=dev)
        for b in range(B):  # one batch element at a time keeps the float raster small
            Sb = (torch.rand((C_in, T), generator=g, device=dev) < prob[b]).to(torch.float32)
            words[b] = alif.pack_spikes(Sb)
        net = network.ALIFNet(C_in, H, K, dt=dt, arp=2.0, device=dev)
        y = labels.to(torch.int32)

        def step():
            for prm in net.parameters():
                prm.grad = None
            loss = net.loss(words, y, T)
            loss.backward()
            return loss
        step()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            loss = step()
        e1.record()
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / steps
        ns = B * sum(H) * T
        out[f"T{T}_dt{dt:g}"] = {"ms_per_step": ms, "neuron_steps_per_s": ns / (ms / 1e3),
                                 "loss": float(loss.detach()), "T_R": alif.tr(dt, 2.0)}
        del net, words
    out["workload"] = ("classification training step: 700 Poisson channels (20 class rate profiles) -> "
                       "256 ALIF -> 256 ALIF -> 20 leaky readout, CE, B=128, fwd+bwd via autograd")
    return out


def seq_fwd_bwd(alif, I, table, spikes, gS, vtr, atr, fin, ws, gI, gp, want_gI=True):
    """The plain step-by-step training pass: forward saving the V/a traces its backward reads,
    then the backward (one thread per row, a loop over t, FP32)."""
    alif.forward_into(I, table, spikes, v=vtr, a=atr, final=fin, seq=True)
    alif.backward(I, table, spikes, gS, v_trace=vtr, a_trace=atr, seq=True, workspace=ws,
                  out_gI=gI if want_gI else None, want_gI=want_gI, out_gp=gp)


def sweep_config(dev, reps=3):
    """Speed-up sweep of the feedforward layer (B=32, N=1024): T in {1000, 4000, 16000} x
    ARP in {1, 2, 4} ms at DT=0.1 ms (T_R 10/20/40).  Currents are precomputed (the projection
    does not depend on T_R); per point the blocked forward, blocked backward and the plain
    sequential forward (spikes and final state only) on the same currents."""
    import torch
    from paper_2311_11390_gb300 import alif, synth
    B, N, Nin = 32, WORKLOAD["N"], WORKLOAD["Nin"]
    out = []
    for T in (1000, 4000, 16000):
        w = synth.feedforward(seed=0, B=B, Nin=Nin, N=N, T=T, dt=WORKLOAD["dt"], arp=2.0)
        Wd = torch.from_numpy(w.W).to(dev)
        hi, lo = alif.split_bf16(Wd)
        S = torch.from_numpy(synth.pack_bits(w.S_in).view(np.int32)).to(dev)
        I = alif.syn_project(S, hi, lo, torch.from_numpy(w.bias).to(dev), Nin=Nin, T=T)
        g = torch.Generator(device=dev).manual_seed(3)
        gS = torch.randn(I.shape, device=dev, generator=g)
        ws = torch.empty(alif.workspace_size(B, N), dtype=torch.uint8, device=dev)
        spikes = torch.empty((B, N, (T + 31) // 32), dtype=torch.int32, device=dev)
        ckpt = torch.empty((B, N, alif.ckpt_count(T), 3), dtype=torch.int32, device=dev)
        fin = torch.empty((B, N, 3), dtype=torch.int32, device=dev)
        gI = torch.empty_like(I)
        vtr, atr = torch.empty_like(I), torch.empty_like(I)
        gp = torch.empty((5, N), device=dev, dtype=torch.float32)
        for arp in (1.0, 2.0, 4.0):
            table = alif.neuron_table(w.params.tau_mem, w.params.tau_adapt, w.params.theta0, w.params.d,
                                      w.params.R, w.dt, arp, device=dev)

            def timed(fn):
                fn()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(reps):
                    fn()
                e1.record()
                torch.cuda.synchronize(dev)
                return e0.elapsed_time(e1) / reps
            f = timed(lambda: alif.forward_into(I, table, spikes, ckpt=ckpt, final=fin))
            b = timed(lambda: alif.backward(I, table, spikes, gS, ckpt=ckpt, workspace=ws, out_gI=gI, out_gp=gp))
            sq = timed(lambda: alif.forward_into(I, table, spikes, final=fin, seq=True))
            stg = timed(lambda: alif.forward_into(I, table, spikes, final=fin, seq="staged"))
            sfb = timed(lambda: seq_fwd_bwd(alif, I, table, spikes, gS, vtr, atr, fin, ws, gI, gp))
            n = B * N * T
            out.append({"T": T, "arp_ms": arp, "T_R": alif.tr(WORKLOAD["dt"], arp), "fwd_ms": f, "bwd_ms": b,
                        "seq_fwd_ms": sq, "staged_seq_fwd_ms": stg, "seq_fwd_bwd_ms": sfb,
                        "fwd_neuron_steps_per_s": n / (f / 1e3),
                        "blocked_over_sequential_fwd": sq / f, "blocked_over_staged_fwd": stg / f,
                        "blocked_over_sequential_fwd_bwd": sfb / (f + b)})
        del I, gS, gI, vtr, atr
    return out


def population_config(dev, reps=20):
    """The small single-population case (B=8, N=128, T=1000, DT=0.1 ms, T_R=20): launch-bound,
    reported for completeness (forward and forward+backward)."""
    import torch
    from paper_2311_11390_gb300 import alif, synth
    w = synth.population(seed=0)
    I = torch.from_numpy(w.I).to(dev)
    table = alif.neuron_table(w.params.tau_mem, w.params.tau_adapt, w.params.theta0, w.params.d,
                              w.params.R, w.dt, w.arp, device=dev)
    B, N, T = I.shape
    spikes = torch.empty((B, N, (T + 31) // 32), dtype=torch.int32, device=dev)
    ckpt = torch.empty((B, N, alif.ckpt_count(T), 3), dtype=torch.int32, device=dev)
    g = torch.Generator(device=dev).manual_seed(0)
    gS = torch.randn(I.shape, device=dev, generator=g)
    ws = torch.empty(alif.workspace_size(B, N), dtype=torch.uint8, device=dev)
    gI = torch.empty_like(I)
    gp = torch.empty((5, N), device=dev, dtype=torch.float32)

    def fb():
        alif.forward_into(I, table, spikes, ckpt=ckpt)
        alif.backward(I, table, spikes, gS, ckpt=ckpt, workspace=ws, out_gI=gI, out_gp=gp)
    vtr, atr = torch.empty_like(I), torch.empty_like(I)
    fin = torch.empty((B, N, 3), dtype=torch.int32, device=dev)
    res = {}
    for name, fn in (("fwd", lambda: alif.forward_into(I, table, spikes, ckpt=ckpt)), ("fwd_bwd", fb),
                     ("seq_fwd", lambda: alif.forward_into(I, table, spikes, final=fin, seq=True)),
                     ("staged_seq_fwd", lambda: alif.forward_into(I, table, spikes, final=fin, seq="staged")),
                     ("seq_fwd_bwd", lambda: seq_fwd_bwd(alif, I, table, spikes, gS, vtr, atr, fin, ws, gI, gp))):
        fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / reps
        res[name + "_ms"] = ms
        res[name + "_neuron_steps_per_s"] = B * N * T / (ms / 1e3)
    res["blocked_over_sequential_fwd"] = res["seq_fwd_ms"] / res["fwd_ms"]
    res["blocked_over_staged_fwd"] = res["staged_seq_fwd_ms"] / res["fwd_ms"]
    res["blocked_over_sequential_fwd_bwd"] = res["seq_fwd_bwd_ms"] / res["fwd_bwd_ms"]
    res["workload"] = "single population B=8 N=128 T=1000 DT=0.1 ms T_R=20, bias U[0.8,1.6] + N(0, 0.3^2)"
    return res


def dt_reference():
    """Fine-DT reference spike steps of the sweep's sample neurons, written by the FP64 oracle
    (tests/golden/make_dt_sweep_reference.py); read here as data."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests", "golden", "dt_sweep_reference.txt")
    out = []
    for line in open(path):
        if line.startswith("#") or "|" not in line:
            continue
        out.append([int(x) for x in line.split("|")[1].split()])
    return out


def dt_sweep_config(dev, reps=3):
    """Speed-accuracy trade-off over DT (the paper's motivating figure): 1024 neurons with
    fit-like parameters driven by one Ornstein-Uhlenbeck current drawn at DT = 0.01 ms for 1 s
    (synth.dt_sweep).  For each DT the current is averaged over its bins and the blocked forward
    is timed on all 1024 neurons.  Accuracy: the spike trains of the first 32 neurons, placed at
    the end of their bins on the 0.01 ms grid, against the FP64 oracle's 0.01 ms trains of the
    same neurons (squared van Rossum distance, tau 5 ms, computed by the library kernel)."""
    import torch
    from paper_2311_11390_gb300 import alif, synth
    w = synth.dt_sweep()
    n, fine, Tf = w.params.N, w.fine_dt, w.x_fine.size
    ref_steps = dt_reference()
    ns = len(ref_steps)
    ref_S = np.zeros((ns, Tf), np.uint8)
    for i, st in enumerate(ref_steps):
        ref_S[i, st] = 1
    ref_words = torch.from_numpy(synth.pack_bits(ref_S).view(np.int32)).to(dev)
    p = w.params
    out = []
    for dt in (0.01, 0.02, 0.05, 0.1, 0.2, 0.5, 1.0):
        f = int(round(dt / fine))
        x = torch.from_numpy(synth.bin_current(w.x_fine, f)).to(dev)
        T = x.numel()
        I = x[None, None, :].expand(1, n, T).contiguous()
        table = alif.neuron_table(p.tau_mem, p.tau_adapt, p.theta0, p.d, p.R, dt, 2.0, device=dev)
        res = alif.forward(I, table, want_ckpt=False)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            res = alif.forward(I, table, want_ckpt=False)
        e1.record()
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / reps
        S = alif.unpack_spikes(res["spikes"][0, :ns], T).cpu().numpy()
        words = torch.from_numpy(synth.pack_bits(synth.place_on_fine_grid(S, f)).view(np.int32)).to(dev)
        loss = torch.empty(ns, device=dev)
        alif.vanrossum_forward(words, ref_words, Tf, fine, 5.0, 256 * ((Tf + 255) // 256), loss=loss)
        out.append({"dt_ms": dt, "T_R": alif.tr(dt, 2.0), "fwd_ms": ms,
                    "simulated_s_per_wall_s": n * w.seconds / (ms / 1e3),
                    "van_rossum_sq_vs_oracle": float(loss.mean()),
                    "spike_count_ratio_vs_oracle": float(S.sum()) / max(float(ref_S.sum()), 1.0)})
        del I
    return {"workload": f"{n} neurons, 1 OU current (tau 3 ms), {w.seconds} s, ARP 2 ms; accuracy of neurons "
                        f"0..{ns - 1} against the FP64 oracle at DT = {fine} ms", "points": out}


def recurrent_line(alif, dev, stream, world, I_ff, table, gS, ws, gI, gp, kern_ms, w, B, N, T, reps=3):
    """The bench workload with recurrent synapses W_rec ~ N(0, 1.5^2 / N) and latency D = T_R
    (Section 2, Prop 3): recurrent forward on the projection's current, then the detached
    backward on the total current and dL/dW_rec against the spikes delayed by T_R."""
    import torch
    TR = alif.tr(w.dt, w.arp)
    rng = np.random.default_rng(5)
    W_rec = torch.from_numpy((1.5 * rng.standard_normal((N, N)) / np.sqrt(N)).astype(np.float32)).to(dev)
    Wt_rec = alif.transpose_weights(W_rec)
    I_tot = torch.empty_like(I_ff)
    state = {}

    def fwd():
        state["r"] = alif.forward_recurrent(I_ff, Wt_rec, table, w.dt, w.arp, out_I=I_tot, want_final=False)

    def bwd():
        r = state["r"]
        alif.backward(I_tot, table, r["spikes"], gS, ckpt=r["ckpt"], workspace=ws, out_gI=gI, out_gp=gp)
        alif.syn_project_backward(alif.delay_spikes(r["spikes"], T, TR), gI, Nin=N, want_gb=False)

    fwd()
    bwd()
    torch.cuda.synchronize(dev)
    assert alif.device_status(dev) == 0
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    f_ms, s_ms = [], []
    for _ in range(reps):
        e[0].record(stream)
        fwd()
        e[1].record(stream)
        bwd()
        e[2].record(stream)
        torch.cuda.synchronize(dev)
        f_ms.append(e[0].elapsed_time(e[1]))
        s_ms.append(e[0].elapsed_time(e[2]))
    f = max_over_ranks(min(f_ms), world, dev)
    st = max_over_ranks(min(s_ms), world, dev) + kern_ms.get("syn_project", 0.0)
    nsp = float(alif.unpack_spikes(state["r"]["spikes"][:1], T).sum()) / N / (T * w.dt * 1e-3)
    units = B * N * T
    return {"workload": f"bench workload + W_rec [{N}x{N}] ~ N(0, 1.5^2/{N}), latency D = T_R = {TR} "
                        f"({(T + TR - 1) // TR} spike exchanges per batch element)",
            "forward_ms": f, "fwd_value": units * world / (f / 1e3),
            "step_ms": st, "value": units * world / (st / 1e3),
            "step": "feedforward projection + recurrent forward + detached backward on the total current + dL/dW_rec",
            "rate_hz_batch0": nsp}


# ------------------------------------------------------------- GPU arm
def targets_summary(line) -> dict:
    """The method's targets in one compact object: speed-ups of the blocked kernels over the
    plain step-by-step kernels as [fwd vs plain, fwd vs staged, fwd+bwd vs plain] for the
    single population (B=8, N=128, T=1000), each T x T_R point of the feedforward layer and
    the neuron fit (T=400000, T_R=40); the HBM fraction of the forward and backward kernels
    (on their own algorithmic bytes and on those of a per-Block saved state); serving latency."""
    r2 = lambda x: None if x is None else round(float(x), 2)
    t = {"key": "[blocked/plain fwd, blocked/staged fwd, blocked/plain fwd+bwd]"}
    pop = line.get("population")
    if pop:
        t["pop_B8_N128_T1000_TR20"] = [r2(pop.get("blocked_over_sequential_fwd")),
                                       r2(pop.get("blocked_over_staged_fwd")),
                                       r2(pop.get("blocked_over_sequential_fwd_bwd"))]
    for p in line.get("sweep") or []:
        t[f"ff_B32_T{p['T']}_TR{p['T_R']}"] = [r2(p.get("blocked_over_sequential_fwd")),
                                               r2(p.get("blocked_over_staged_fwd")),
                                               r2(p.get("blocked_over_sequential_fwd_bwd"))]
    fit = line.get("fit")
    if fit and "blocked_over_sequential_fwd" in fit:
        t["fit_N1024_T400000_TR40"] = [r2(fit.get("blocked_over_sequential_fwd")),
                                       r2(fit.get("blocked_over_staged_fwd")),
                                       r2(fit.get("blocked_over_sequential_fwd_bwd"))]
    hf = (line.get("roofline") or {}).get("hbm_frac") or {}
    t["hbm_frac"] = {k: round(v, 3) for k, v in hf.items()}
    hs = (line.get("roofline") or {}).get("hbm_frac_per_block_state") or {}
    t["hbm_frac_per_block_state"] = {k: round(v, 3) for k, v in hs.items()}
    srv = line.get("serve")
    if srv:
        t["serve"] = {"requests": srv.get("requests"), "p50_ms": r2(srv.get("p50_ms")), "p99_ms": r2(srv.get("p99_ms")),
                      "neuron_steps_per_s": float("%.3g" % srv["neuron_steps_per_s"])}
    e2e = line.get("e2e")
    if e2e:
        t["e2e_ms"] = r2(e2e["ms_per_step"])
    fu = line.get("fused_projection_forward")
    if fu:
        t["fused_vs_separate_ms"] = [r2(fu["kernel_ms"]), r2(fu["separate_ms"])]
    return t


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2311_11390_gb300 import alif
    from paper_2311_11390_gb300.pipeline import DoubleBuffered

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    L = alif.lib()
    has_proj = getattr(L, "syn_project", None) is not None
    B, T, N, Nin = args.B, args.T, WORKLOAD["N"], WORKLOAD["Nin"]
    w, packed = make_inputs(rank, B, T, args.arp)
    table = alif.neuron_table(w.params.tau_mem, w.params.tau_adapt, w.params.theta0, w.params.d,
                              w.params.R, w.dt, w.arp, device=dev)
    S_dev = torch.from_numpy(packed.view(np.int32)).to(dev)
    W_dev = torch.from_numpy(w.W).to(dev)
    bias = torch.from_numpy(w.bias).to(dev)
    g = torch.Generator(device=dev).manual_seed(1234 + rank)
    gS = torch.randn((B, N, T), device=dev, generator=g, dtype=torch.float32)
    ws = torch.empty(alif.workspace_size(B, N), dtype=torch.uint8, device=dev)
    nwords = (T + 31) // 32
    I = torch.empty((B, N, T), device=dev, dtype=torch.float32)
    gI = torch.empty_like(I)
    spikes = torch.empty((B, N, nwords), device=dev, dtype=torch.int32)
    ckpt = torch.empty((B, N, alif.ckpt_count(T), 3), device=dev, dtype=torch.int32)
    fin = torch.empty((B, N, 3), device=dev, dtype=torch.int32)
    gp = torch.empty((5, N), device=dev, dtype=torch.float32)
    if has_proj:
        Whi, Wlo = alif.split_bf16(W_dev)
    else:  # library without the projection: currents computed once, outside the timed step
        for b in range(B):
            Sb = torch.from_numpy(w.S_in[b]).to(dev, dtype=torch.float32)
            I[b] = W_dev @ Sb + bias[:, None]
    stream = torch.cuda.current_stream(dev)
    names = ["syn_project", "alif_forward", "alif_backward"]
    ev = {n: [] for n in names}

    def step(record=False):
        marks = []
        if has_proj:
            e0 = torch.cuda.Event(enable_timing=True) if record else None
            if record:
                e0.record(stream)
            alif.syn_project(S_dev, Whi, Wlo, bias, Nin=Nin, T=T, out=I)
            if record:
                marks.append(("syn_project", e0))
        e1 = torch.cuda.Event(enable_timing=True) if record else None
        if record:
            e1.record(stream)
        alif.forward_into(I, table, spikes, ckpt=ckpt, final=fin)
        e2 = torch.cuda.Event(enable_timing=True) if record else None
        if record:
            e2.record(stream)
        alif.backward(I, table, spikes, gS, ckpt=ckpt, workspace=ws, out_gI=gI, out_gp=gp)
        e3 = torch.cuda.Event(enable_timing=True) if record else None
        if record:
            e3.record(stream)
            if has_proj:
                ev["syn_project"].append((marks[0][1], e1))
            ev["alif_forward"].append((e1, e2))
            ev["alif_backward"].append((e2, e3))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    assert alif.device_status(dev) == 0
    barrier(world)
    torch.cuda.synchronize(dev)
    with ClockSampler(local_rank) as clk:
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for _ in range(args.steps):
            step(record=True)
        t_end.record(stream)
        torch.cuda.synchronize(dev)
    barrier(world)
    ms_total = t_start.elapsed_time(t_end)
    ms_total = max_over_ranks(ms_total, world, dev)
    ms_step = ms_total / args.steps
    steps_per_rank = B * N * T
    value = steps_per_rank * world / (ms_step / 1e3)
    kern_ms = {n: statistics.mean(a.elapsed_time(b) for a, b in ev[n]) for n in names if ev[n]}
    launches_per_step = (1 if has_proj else 0) + 1 + 2  # projection, forward, backward + batch reduction

    # ---- roofline of the dominant kernel (algorithmic bytes or flops per launch)
    pk, pk_kind = peaks()
    alg = {
        "alif_forward": ("hbm", steps_per_rank * (4 + 1 / 8 + 12 / 256)),
        "alif_backward": ("hbm", steps_per_rank * (4 + 4 + 4 + 1 / 8 + 12 / 256)),
        # dense split-BF16 contraction: 2 flops x 2 terms per weight and (b, t)
        "syn_project": ("tensor", 4.0 * N * Nin * T * B),
    }
    dom = max(kern_ms, key=kern_ms.get)
    bound, work = alg[dom]
    if bound == "hbm":
        achieved, peak, unit = work / (kern_ms[dom] / 1e3) / 1e9, pk["hbm_gbs"], "GB/s"
    else:
        achieved = work / (kern_ms[dom] / 1e3) / 1e12
        peak, unit = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops")), "TFLOP/s"
    roof = {"kernel": dom, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": achieved / peak, "traffic": profiled_traffic(dom, steps_per_rank), "peak_kind": pk_kind,
            "work_per_launch": work, "kernel_ms": kern_ms,
            "hbm_frac": {k: (alg[k][1] / (kern_ms[k] / 1e3) / 1e9) / pk["hbm_gbs"]
                         for k in kern_ms if alg[k][0] == "hbm"}}
    # the same fractions on the bytes of a layout that saves a 9-byte state at every Block (9 / T_R
    # per neuron-step) instead of the 12-byte checkpoint every 256 steps these kernels write, and
    # whose backward reads no spike bits
    TR = alif.tr(w.dt, w.arp)
    alg_s = {"alif_forward": steps_per_rank * (4 + 1 / 8 + 9 / TR), "alif_backward": steps_per_rank * (12 + 9 / TR)}
    roof["hbm_frac_per_block_state"] = {k: (alg_s[k] / (kern_ms[k] / 1e3) / 1e9) / pk["hbm_gbs"] for k in kern_ms
                                     if k in alg_s}

    # ---- the event-driven projection on the same step (a separate line; the step above
    # keeps the tensor-core projection)
    extra = {}
    if has_proj and getattr(L, "syn_project_events", None) is not None:
        Wt_dev = alif.transpose_weights(W_dev)
        I_ev = torch.empty_like(I)
        alif.syn_project_events(S_dev, Wt_dev, bias, Nin=Nin, T=T, out=I_ev)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 5
        e0.record(stream)
        for _ in range(reps):
            alif.syn_project_events(S_dev, Wt_dev, bias, Nin=Nin, T=T, out=I_ev)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ev_ms = max_over_ranks(e0.elapsed_time(e1) / reps, world, dev)
        step_ev = ev_ms + kern_ms["alif_forward"] + kern_ms["alif_backward"]
        extra["event_projection"] = {
            "kernel_ms": ev_ms, "tensor_core_kernel_ms": kern_ms["syn_project"],
            "hbm_frac_of_output_write": (steps_per_rank * 4 / (ev_ms / 1e3) / 1e9) / pk["hbm_gbs"],
            "step_ms": step_ev, "value": steps_per_rank * world / (step_ev / 1e3),
            "kernel": "event-driven: bias + sum of the active inputs' FP32 weights, per (batch, 32-step chunk) "
                      "event lists in shared memory, deterministic order"}
        del I_ev, Wt_dev

    # ---- the projection fused into the block forward (currents summed inside the forward from the
    # input events, written for the backward): a separate line beside the step's two kernels
    if has_proj and getattr(L, "alif_forward_fused", None) is not None and Nin <= 1024:
        cap = 1024  # events per (batch element, 32-step word); an overflow would fail the status check below
        fws = torch.empty(int(L.alif_forward_fused_workspace_size(B, Nin, T, cap)), dtype=torch.uint8, device=dev)
        I_fu = torch.empty_like(I)

        def fused():
            alif.forward_fused(S_dev, W_dev, bias, table, T, max_events_per_word=cap, out_I=I_fu, out_spikes=spikes,
                               out_ckpt=ckpt, out_final=fin, workspace=fws)
        fused()
        torch.cuda.synchronize(dev)
        assert alif.device_status(dev) == 0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            fused()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        fu_ms = max_over_ranks(e0.elapsed_time(e1) / 3, world, dev)
        extra["fused_projection_forward"] = {
            "kernel_ms": fu_ms, "separate_ms": kern_ms["syn_project"] + kern_ms["alif_forward"],
            "events_separate_ms": (extra.get("event_projection") or {}).get("kernel_ms", float("nan")) + kern_ms["alif_forward"],
            "max_events_per_word": cap,
            "kernel": "event buckets of the raster, then the block forward summing each step's active weights "
                      "(FP32 weight row in shared memory) and writing the currents for the backward"}
        del I_fu, fws

    # ---- projection backward (dL/dW and dL/dbias, event-driven) on the step's dL/dI: a separate
    # line; the headline step trains the neurons and stops at dL/dI
    if has_proj and getattr(L, "syn_project_backward", None) is not None:
        alif.syn_project_backward(S_dev, gI, Nin=Nin, want_gW=True, want_gb=True)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 3
        e0.record(stream)
        for _ in range(reps):
            alif.syn_project_backward(S_dev, gI, Nin=Nin, want_gW=True, want_gb=True)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        pb_ms = max_over_ranks(e0.elapsed_time(e1) / reps, world, dev)
        pb_bytes = B * N * T * 4 + B * Nin * ((T + 31) // 32) * 4 + N * Nin * 4 + N * 4
        extra["projection_backward"] = {
            "kernel_ms": pb_ms, "algorithmic_bytes": pb_bytes,
            "achieved_gbs": pb_bytes / (pb_ms / 1e3) / 1e9,
            "hbm_frac": pb_bytes / (pb_ms / 1e3) / 1e9 / pk["hbm_gbs"],
            "input_spikes": int(w.S_in.sum()),
            "kernel": "dL/dW = sum_b,t dL/dI S^T and dL/dbias, event-driven (per batch element and 16-row "
                      "tile, dL/dI staged step-major in 512-step chunks, one thread per input walking its "
                      "spikes and adding the staged columns in registers), partials summed over the batch "
                      "in a fixed order"}

    # ---- the same workload as a recurrent layer (W_rec, latency D = T_R): a separate line
    if has_proj and not args.no_rec and getattr(L, "alif_forward_recurrent", None) is not None:
        extra["recurrent"] = recurrent_line(alif, dev, stream, world, I, table, gS, ws, gI, gp, kern_ms, w, B, N, T)

    # ---- forward-only and the plain sequential kernels on the same inputs
    fwd_value = steps_per_rank / (kern_ms["alif_forward"] / 1e3)
    extra["fwd_value"] = fwd_value * world
    if not args.no_seq:
        vtr = torch.empty_like(I)
        atr = torch.empty_like(I)

        def seq_step():
            alif.forward_into(I, table, spikes, v=vtr, a=atr, final=fin, seq=True)
            alif.backward(I, table, spikes, gS, v_trace=vtr, a_trace=atr, seq=True, workspace=ws, out_gI=gI,
                          out_gp=gp)
        seq_step()
        torch.cuda.synchronize(dev)
        reps = 2
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a2 = torch.cuda.Event(enable_timing=True)

        def timed(fn):
            fn()
            ts = []
            for _ in range(reps):
                a0.record(stream)
                fn()
                a1.record(stream)
                torch.cuda.synchronize(dev)
                ts.append(a0.elapsed_time(a1))
            return min(ts)
        # forward only, spikes + final state (what the blocked forward's line produces, minus ckpt)
        seq_f = timed(lambda: alif.forward_into(I, table, spikes, final=fin, seq=True))
        stg_f = timed(lambda: alif.forward_into(I, table, spikes, final=fin, seq="staged"))
        fw, fb = [], []
        for _ in range(reps):  # forward with the traces its backward needs, then the backward
            a0.record(stream)
            alif.forward_into(I, table, spikes, v=vtr, a=atr, final=fin, seq=True)
            a1.record(stream)
            alif.backward(I, table, spikes, gS, v_trace=vtr, a_trace=atr, seq=True, workspace=ws, out_gI=gI,
                          out_gp=gp)
            a2.record(stream)
            torch.cuda.synchronize(dev)
            fw.append(a0.elapsed_time(a1))
            fb.append(a0.elapsed_time(a2))
        seq_fb = min(fb)
        blk_fb = kern_ms["alif_forward"] + kern_ms["alif_backward"]
        extra["sequential"] = {
            "fwd_value": steps_per_rank * world / (seq_f / 1e3),
            "fwd_bwd_value": steps_per_rank * world / (seq_fb / 1e3),
            "blocked_over_sequential_fwd": seq_f / kern_ms["alif_forward"],
            "blocked_over_sequential_fwd_bwd": seq_fb / blk_fb,
            "kernel": "one thread per (b, i), per-step loop over t, FP32; forward-only line writes spikes "
                      "and the final state, the fwd+bwd line saves V/a traces for its backward",
            "staged_fwd_value": steps_per_rank * world / (stg_f / 1e3),
            "blocked_over_staged_fwd": stg_f / kern_ms["alif_forward"],
            "staged_kernel": "same recurrence, input staged through shared memory in coalesced "
                             "32-row x 32-step tiles with the next tile prefetched (honesty line)"}

    # ---- end to end through the public API with host buffers.  Every step uploads its inputs
    # from pinned host memory (the input spike raster and the upstream gradient dL/dS) and
    # downloads its results (output spikes, dL/dI and the parameter gradients); two slots of
    # device buffers let step k's copies overlap steps k-1 and k+1's compute.  A second line
    # moves only the spikes in and the spikes and parameter gradients out (dL/dS and dL/dI
    # resident on the device).
    e2e = e2e_spikes = None
    if has_proj:
        S_host = torch.from_numpy(packed.view(np.int32)).pin_memory()
        gS_host = torch.empty(gS.shape, dtype=torch.float32).pin_memory()
        gS_host.copy_(gS)
        spk_host = [torch.empty(spikes.shape, dtype=torch.int32).pin_memory() for _ in range(2)]
        gp_host = [torch.empty(gp.shape, dtype=torch.float32).pin_memory() for _ in range(2)]

        def run_e2e(with_grads: bool, reps: int):
            if with_grads:
                gI_host = [torch.empty(gI.shape, dtype=torch.float32).pin_memory() for _ in range(2)]

            def make_slot():
                sl = {"S": torch.empty_like(S_dev), "spikes": torch.empty_like(spikes), "gp": torch.empty_like(gp)}
                if with_grads:
                    sl["gS"], sl["gI"] = torch.empty_like(gS), torch.empty_like(gI)
                return sl
            pipe = DoubleBuffered(dev, make_slot)

            def load(k, sl):
                sl["S"].copy_(S_host, non_blocking=True)
                if with_grads:
                    sl["gS"].copy_(gS_host, non_blocking=True)

            def compute(k, sl):
                g_in = sl["gS"] if with_grads else gS
                g_out = sl["gI"] if with_grads else gI
                alif.syn_project(sl["S"], Whi, Wlo, bias, Nin=Nin, T=T, out=I)
                alif.forward_into(I, table, sl["spikes"], ckpt=ckpt, final=fin)
                alif.backward(I, table, sl["spikes"], g_in, ckpt=ckpt, workspace=ws, out_gI=g_out, out_gp=sl["gp"])

            def store(k, sl):
                spk_host[k & 1].copy_(sl["spikes"], non_blocking=True)
                gp_host[k & 1].copy_(sl["gp"], non_blocking=True)
                if with_grads:
                    gI_host[k & 1].copy_(sl["gI"], non_blocking=True)

            pipe.run(2, load, compute, store, stream=stream)  # untimed: first use of the slots
            torch.cuda.synchronize(dev)
            e_s = torch.cuda.Event(enable_timing=True)
            e_e = torch.cuda.Event(enable_timing=True)
            e_s.record(stream)
            pipe.run(reps, load, compute, store, stream=stream)
            e_e.record(stream)
            torch.cuda.synchronize(dev)
            ms = max_over_ranks(e_s.elapsed_time(e_e) / reps, world, dev)
            h2d = S_host.numel() * 4 + (gS_host.numel() * 4 if with_grads else 0)
            d2h = spk_host[0].numel() * 4 + gp_host[0].numel() * 4 + (gI.numel() * 4 if with_grads else 0)
            del pipe
            return {"value": steps_per_rank * world / (ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h), "ms_per_step": ms, "steps": reps}

        # a stream of up to 20 steps: the first step's upload and the last one's download have no
        # neighbour to overlap with, and longer streams amortise that fill and drain
        e2e = run_e2e(True, max(4, min(args.steps, 20)))
        e2e["copies"] = ("per step: input spike raster and dL/dS host -> device, output spikes, dL/dI and "
                         "parameter gradients device -> host; pinned host buffers, one copy per tensor on "
                         "two copy streams, double-buffered device slots overlapping the compute")
        e2e_spikes = run_e2e(False, max(4, min(args.steps, 10)))
        e2e_spikes["copies"] = ("per step: input spike raster in, output spikes and parameter gradients out; "
                                "dL/dS and dL/dI stay on the device")
        del gS_host

    # ---- CPU oracle baseline (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        from oracle import ref
        ref.build()
        cores = os.cpu_count() or 1
        rows = 512
        n, s = cpu_oracle_sample(w, rows, cores)
        cpu = {"value": n / s, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"batch element 0, neurons 0..{rows - 1}, full T={T}: FP64 projection + "
                         f"step-by-step forward + BPTT, {cores} threads over rows"}

    if rank == 0 and world == 1 and not args.no_fit:
        extra["fit"] = fit_config(dev, with_seq=not args.no_seq)
    if rank == 0 and world == 1 and not args.no_serve:
        extra["serve"] = serve_config(dev, args.serve_requests)
    if rank == 0 and world == 1 and not args.no_train:
        extra["train"] = train_config(dev, Ts=tuple(args.train_T))
    if rank == 0 and world == 1 and not args.no_sweep:
        extra["sweep"] = sweep_config(dev)
        extra["population"] = population_config(dev)
        extra["dt_sweep"] = dt_sweep_config(dev)
    assert alif.device_status(dev) == 0
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded Poisson inputs)",
            "config": {"workload": "feedforward ALIF layer: 1000 Poisson inputs -> N=1024, B=%d per GPU, "
                                   "T=%d, DT=0.1 ms, ARP=%g ms (T_R=%d)" % (B, T, args.arp, alif.tr(0.1, args.arp)),
                       "global_batch": B * world, "seq_len": T, "parallelism": f"dp{world} (independent rows)",
                       "l2": "inputs larger than L2 (I, dL/dS: %.1f GB each)" % (steps_per_rank * 4 / 1e9),
                       "projection": "tcgen05 split-BF16" if has_proj else "not in the loaded library (currents precomputed)"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "e2e_spikes_only": e2e_spikes, "gpu_launches": launches_per_step * args.steps,
            "clocks": clk.summary(), **extra}
    line["targets"] = targets_summary(line)  # last, so the end of the printed line carries it
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local_rank = dist_env()
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend=backend)
    try:
        if args.impl == "reference":
            run_reference(args, rank, world)
        else:
            run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
