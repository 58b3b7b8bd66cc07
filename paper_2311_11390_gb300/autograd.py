"""torch.autograd integration of the block forward / backward.

`ALIFFunction` runs the blocked forward and saves only what the backward needs:
the input current I (a reference, not a copy), the bit-packed spikes and the
block-boundary states (one AlifState per 256 steps).  Its backward is the
hand-written surrogate-gradient kernel (fast sigmoid by default; detached reset
and adaptation by default, "attached" on request), which recomputes V and a
inside each window.  The per-neuron
parameters are plain tensors; their FP64 preparation (beta = exp(-DT/tau) ...)
runs on the host when their values change.
"""
from __future__ import annotations

import numpy as np
import torch

from . import alif

_TABLES: dict = {}


def _table(tau_mem, tau_adapt, theta0, d, R, dt, arp, device):
    """Prepared neuron table for the current parameter values (cached by version)."""
    key = tuple((t.data_ptr(), t._version) if t is not None else None
                for t in (tau_mem, tau_adapt, theta0, d, R)) + (float(dt), float(arp), str(device))
    tab = _TABLES.get(key)
    if tab is None:
        host = [None if t is None else t.detach().to("cpu", torch.float32).numpy()
                for t in (tau_mem, tau_adapt, theta0, d, R)]
        tab = torch.from_numpy(alif.prepare(*host, dt_ms=dt, arp_ms=arp)).to(device)
        if len(_TABLES) > 64:
            _TABLES.clear()
        _TABLES[key] = tab
    return tab


class ALIFFunction(torch.autograd.Function):
    """(S, words) = ALIF(I; tau_mem, tau_adapt, theta0, d, R).  I: float32 [B, N, T] on the GPU.
    S is the spike train as float32 0/1 [B, N, T] (differentiable through the surrogate);
    words are the same spikes as int32 bits [B, N, ceil(T/32)] (not differentiable), the
    form the next layer's projection consumes."""

    @staticmethod
    def forward(ctx, I, tau_mem, tau_adapt, theta0, d, R, dt, arp, slope, surrogate="fast_sigmoid",
                attached=False):
        I = I.contiguous()
        table = _table(tau_mem, tau_adapt, theta0, d, R, dt, arp, I.device)
        out = alif.forward(I, table, want_ckpt=True, want_final=False)
        S = alif.spikes_to_float(out["spikes"], I.shape[-1])
        ctx.save_for_backward(I, out["spikes"], out["ckpt"], table)
        ctx.slope = float(slope)
        ctx.surrogate = surrogate
        ctx.attached = bool(attached)
        ctx.has_R = R is not None
        ctx.param_meta = [(t.dtype, t.device) if t is not None else None
                          for t in (tau_mem, tau_adapt, theta0, d, R)]
        words = out["spikes"]
        ctx.mark_non_differentiable(words)
        return S, words

    @staticmethod
    def backward(ctx, grad_S, _grad_words=None):
        I, spikes, ckpt, table = ctx.saved_tensors
        grad_S = grad_S.contiguous().to(torch.float32)
        gI, _, gp = alif.backward(I, table, spikes, grad_S, ckpt=ckpt, slope=ctx.slope,
                                  want_gI=ctx.needs_input_grad[0], surrogate=ctx.surrogate,
                                  attached=ctx.attached)
        grads = []
        for k, meta in enumerate(ctx.param_meta):
            if meta is None or not ctx.needs_input_grad[1 + k]:
                grads.append(None)
            else:
                grads.append(gp[k].to(dtype=meta[0], device=meta[1]))
        return (gI, *grads, None, None, None, None, None)


def alif_spikes(I, tau_mem, tau_adapt, theta0, d, R=None, dt=0.1, arp=2.0, slope=25.0, surrogate="fast_sigmoid",
                attached=False):
    """Functional form: spikes (float 0/1) of an ALIF population driven by I [B, N, T]."""
    return ALIFFunction.apply(I, tau_mem, tau_adapt, theta0, d, R, dt, arp, slope, surrogate, attached)[0]


class ALIFLayer(torch.nn.Module):
    """N ALIF neurons with trainable time constants, threshold baseline and adaptation
    scale (initial values as in the paper's classification setup: tau_mem 20 ms,
    tau_adapt 150 ms, d 1.8)."""

    def __init__(self, N, dt=1.0, arp=2.0, tau_mem=20.0, tau_adapt=150.0, theta0=1.0, d=1.8, slope=25.0):
        super().__init__()
        f = lambda v: torch.nn.Parameter(torch.full((N,), float(v)))
        self.tau_mem, self.tau_adapt, self.theta0, self.d = f(tau_mem), f(tau_adapt), f(theta0), f(d)
        self.dt, self.arp, self.slope = dt, arp, slope

    def forward(self, I, with_words=False):
        S, words = ALIFFunction.apply(I, self.tau_mem, self.tau_adapt, self.theta0, self.d, None, self.dt,
                                      self.arp, self.slope)
        return (S, words) if with_words else S
