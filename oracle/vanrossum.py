"""van Rossum distance oracle -- TEST INFRASTRUCTURE ONLY.

Supplementary "Neural fits": D_R^2 = (1/tau_R) int (k*x - k*y)^2 dt with k(t) = H(t) e^{-t/tau_R},
on the DT grid: f[t] = e^{-DT/tau_R} f[t-1] + x[t] - y[t], loss = (DT/tau_R) sum_t f[t]^2, and its
gradient with respect to x by the reverse recursion g[t] = f[t] + e^{-DT/tau_R} g[t+1],
dL/dx[t] = (2 DT/tau_R) g[t].  Plain float64 loops.
"""
from __future__ import annotations

import math

import numpy as np


def forward(x: np.ndarray, y: np.ndarray, dt: float, tau: float):
    """x, y: [rows, T] in {0,1}. Returns (loss [rows], f [rows, T])."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    dec = math.exp(-dt / tau)
    rows, T = x.shape
    f = np.zeros((rows, T))
    for r in range(rows):
        acc = 0.0
        for t in range(T):
            acc = dec * acc + (x[r, t] - y[r, t])
            f[r, t] = acc
    return (dt / tau) * (f ** 2).sum(axis=1), f


def backward(x: np.ndarray, y: np.ndarray, dt: float, tau: float) -> np.ndarray:
    """dL/dx [rows, T]."""
    _, f = forward(x, y, dt, tau)
    dec = math.exp(-dt / tau)
    rows, T = f.shape
    g = np.zeros_like(f)
    for r in range(rows):
        acc = 0.0
        for t in range(T - 1, -1, -1):
            acc = f[r, t] + dec * acc
            g[r, t] = acc
    return (2.0 * dt / tau) * g
