"""Pins of the classification-network oracle pieces (readout, cross-entropy) against
closed forms and identities the mathematics fixes, independent of the oracle's loops."""
import math

import numpy as np

from oracle import network


def test_readout_closed_form():
    """sum_t V_o[t] with V_o[t] = b V_o[t-1] + (1-b) I[t] equals sum_j I[j] (1 - b^(T-j))
    (geometric sum of the impulse response over the remaining steps)."""
    rng = np.random.default_rng(0)
    B, C, T = 3, 5, 37
    I = rng.standard_normal((B, C, T))
    for beta in (0.0, 0.3, 0.95, 0.999):
        o = network.readout_forward(I, beta)
        j = np.arange(T)
        w = 1.0 - beta ** (T - j)
        np.testing.assert_allclose(o, (I * w).sum(-1), rtol=1e-12, atol=1e-12)


def test_readout_constant_input():
    """Constant input x: o = x (T - b (1 - b^T) / (1 - b))."""
    T, beta, x = 50, 0.9, 1.7
    o = network.readout_forward(np.full((1, 1, T), x), beta)
    np.testing.assert_allclose(o[0, 0], x * (T - beta * (1 - beta ** T) / (1 - beta)), rtol=1e-12)


def test_readout_backward_is_adjoint():
    """The readout is linear in I, so <g_o, o(I)> = <readout_backward(g_o), I>."""
    rng = np.random.default_rng(1)
    B, C, T = 2, 4, 29
    for beta in (0.5, 0.97):
        I = rng.standard_normal((B, C, T))
        g_o = rng.standard_normal((B, C))
        lhs = (g_o * network.readout_forward(I, beta)).sum()
        rhs = (network.readout_backward(g_o, beta, T) * I).sum()
        assert abs(lhs - rhs) <= 1e-11 * max(1.0, abs(lhs))


def test_cross_entropy_uniform_and_invariances():
    C = 20
    o = np.zeros((4, C))
    y = np.array([0, 3, 19, 7])
    L, g = network.cross_entropy(o, y)
    assert abs(L - math.log(C)) < 1e-12
    np.testing.assert_allclose(g.sum(1), 0.0, atol=1e-15)
    rng = np.random.default_rng(2)
    o = rng.standard_normal((4, C)) * 3
    L1, g1 = network.cross_entropy(o, y)
    L2, g2 = network.cross_entropy(o + 11.0, y)  # softmax is shift invariant
    assert abs(L1 - L2) < 1e-12
    np.testing.assert_allclose(g1, g2, atol=1e-14)


def test_cross_entropy_gradient_finite_differences():
    rng = np.random.default_rng(3)
    B, C = 3, 6
    o = rng.standard_normal((B, C))
    y = np.array([1, 5, 0])
    _, g = network.cross_entropy(o, y)
    eps = 1e-6
    for b in range(B):
        for c in range(C):
            op, om = o.copy(), o.copy()
            op[b, c] += eps
            om[b, c] -= eps
            fd = (network.cross_entropy(op, y)[0] - network.cross_entropy(om, y)[0]) / (2 * eps)
            assert abs(fd - g[b, c]) < 1e-8


def test_cross_entropy_known_value():
    """Two classes, logits (0, log 3): p = (1/4, 3/4); label 0 costs log 4, label 1 log(4/3)."""
    o = np.array([[0.0, math.log(3.0)], [0.0, math.log(3.0)]])
    L, _ = network.cross_entropy(o, np.array([0, 1]))
    assert abs(L - 0.5 * (math.log(4.0) + math.log(4.0 / 3.0))) < 1e-12
