"""Pins of the van Rossum oracle: closed form of a single spike, the continuous-time limit,
and exact central differences (the loss is quadratic in x)."""
import math

import numpy as np

from oracle import vanrossum


def test_single_spike_closed_form_and_limit():
    dt, tau, T = 0.1, 5.0, 4000
    x = np.zeros((1, T)); x[0, 10] = 1
    loss, _ = vanrossum.forward(x, np.zeros((1, T)), dt, tau)
    dec = math.exp(-dt / tau)
    n = T - 10
    assert abs(loss[0] - (dt / tau) * (1 - dec ** (2 * n)) / (1 - dec * dec)) < 1e-12
    # DT -> 0: (1/tau) int_0^inf e^{-2t/tau} dt = 1/2
    loss_fine, _ = vanrossum.forward(x, np.zeros((1, T)), 0.001, 0.2)
    assert abs(loss_fine[0] - 0.5) < 3e-3
    # identical trains: zero distance
    assert vanrossum.forward(x, x, dt, tau)[0][0] == 0.0


def test_gradient_is_exact_central_difference():
    rng = np.random.default_rng(0)
    x = (rng.random((2, 300)) < 0.1).astype(np.float64)
    y = (rng.random((2, 300)) < 0.1).astype(np.float64)
    g = vanrossum.backward(x, y, 0.2, 3.0)
    for r, t in [(0, 0), (0, 150), (1, 299), (1, 77)]:
        e = np.zeros_like(x); e[r, t] = 0.5
        num = (vanrossum.forward(x + e, y, 0.2, 3.0)[0][r] - vanrossum.forward(x - e, y, 0.2, 3.0)[0][r]) / 1.0
        assert abs(num - g[r, t]) < 1e-9 * max(1.0, abs(g[r, t]))
