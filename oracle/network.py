"""Classification network pieces -- TEST INFRASTRUCTURE ONLY.

The network of the classification experiments (Section 4.2; Supplementary,
"Classification"): input spikes -> dense projection (Eq 3) -> ALIF layer ->
dense projection -> ALIF layer -> leaky readout -> softmax cross-entropy.
The readout is an integrator with the spike and the reset removed, and the
class score is the sum of its membrane over time:
    V_o[t] = beta_o V_o[t-1] + (1 - beta_o) I_o[t],  V_o[-1] = 0,
    o_c    = sum_t V_o[t],
    L      = -(1/B) sum_b log softmax(o_b)[y_b].
Everything here is float64 and written as plain loops over time (the ALIF
layers and the projections are oracle.ref and oracle.project).
"""
from __future__ import annotations

import math

import numpy as np


def readout_forward(I_o: np.ndarray, beta: float) -> np.ndarray:
    """I_o: [B, C, T] readout input current -> o [B, C] (sum over t of the leaky membrane)."""
    I_o = np.asarray(I_o, np.float64)
    B, C, T = I_o.shape
    V = np.zeros((B, C))
    o = np.zeros((B, C))
    for t in range(T):
        V = beta * V + (1.0 - beta) * I_o[..., t]
        o += V
    return o


def readout_backward(g_o: np.ndarray, beta: float, T: int) -> np.ndarray:
    """dL/dI_o [B, C, T] from dL/do [B, C]: reverse of `readout_forward`
    (G[t] = dL/dV_o[t] = g_o + beta G[t+1], dL/dI_o[t] = (1 - beta) G[t])."""
    g_o = np.asarray(g_o, np.float64)
    G = np.zeros_like(g_o)
    g = np.zeros(g_o.shape + (T,))
    for t in range(T - 1, -1, -1):
        G = g_o + beta * G
        g[..., t] = (1.0 - beta) * G
    return g


def cross_entropy(o: np.ndarray, y: np.ndarray):
    """Mean softmax cross-entropy over the batch and its gradient dL/do."""
    o = np.asarray(o, np.float64)
    B, C = o.shape
    loss = 0.0
    g = np.zeros((B, C))
    for b in range(B):
        m = o[b].max()
        e = np.exp(o[b] - m)
        s = e.sum()
        loss += -(o[b, y[b]] - m - math.log(s))
        g[b] = e / s
        g[b, y[b]] -= 1.0
    return loss / B, g / B


def readout_beta(dt: float, tau: float) -> float:
    return math.exp(-dt / tau)
