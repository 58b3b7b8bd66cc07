"""Exact-arithmetic ALIF checker -- TEST INFRASTRUCTURE ONLY.

An independent, pure-Python restatement of the standard ALIF model (Section 2,
Eqs 1-5) in exact rational arithmetic (fractions.Fraction), used to pin the
FP64 C oracle on tiny inputs where floating-point ties cannot occur:

* `simulate` walks Eqs 1-5 one step at a time with rational beta, p, I, R.
* `consistent` re-simulates V and a for a *given* spike train (spikes fixed in
  the reset of Eq 2, the counter of Eq 4 and the update of Eq 5) and reports
  whether that train equals 1{V > theta} at every step (Eq 1).
* `brute_force` enumerates all 2^T spike trains and returns those that are
  self-consistent; the dynamics are deterministic, so exactly one survives.

Shares no code with the C oracle or the CUDA path.
"""
from __future__ import annotations

from fractions import Fraction as F
from itertools import product


def _admitted(last_spike, t, TR):
    # Eq 4: input enters iff the steps since the last spike C >= T_R.
    return last_spike is None or (t - last_spike) >= TR


def simulate(I, beta, p, theta0, d, TR, R=F(1), V0=F(0), S0=0, a0=F(0), last0=None):
    """Exact Eqs 1-5 for one neuron.  I: list of Fractions (paper t = 1..T).
    last0: time of the last spike before t = 1 (0 means a spike at t = 0), or None.
    Returns (S, V, a, theta) lists indexed by t-1."""
    S_out, V_out, a_out, th_out = [], [], [], []
    V_prev, S_prev, a_prev, last = F(V0), S0, F(a0), last0
    if S0:
        last = 0
    for t, It in enumerate(I, start=1):
        a_t = p * a_prev + S_prev
        th = theta0 + d * a_t
        Iin = It if _admitted(last, t, TR) else F(0)
        V_t = (beta * V_prev + (1 - beta) * R * Iin) * (1 - S_prev)
        s = 1 if V_t > th else 0
        if s:
            last = t
        S_out.append(s); V_out.append(V_t); a_out.append(a_t); th_out.append(th)
        V_prev, S_prev, a_prev = V_t, s, a_t
    return S_out, V_out, a_out, th_out


def consistent(S, I, beta, p, theta0, d, TR, R=F(1)):
    """True iff the fixed spike train S satisfies S[t] = 1{V[t] > theta[t]} for all t
    when V, a are driven by S itself (Eqs 1-5, from rest)."""
    V_prev, S_prev, a_prev, last = F(0), 0, F(0), None
    for t, (It, s) in enumerate(zip(I, S), start=1):
        a_t = p * a_prev + S_prev
        th = theta0 + d * a_t
        Iin = It if _admitted(last, t, TR) else F(0)
        V_t = (beta * V_prev + (1 - beta) * R * Iin) * (1 - S_prev)
        if (1 if V_t > th else 0) != s:
            return False
        if s:
            last = t
        V_prev, S_prev, a_prev = V_t, s, a_t
    return True


def brute_force(I, beta, p, theta0, d, TR, R=F(1)):
    """All self-consistent spike trains of length len(I) (2^T candidates)."""
    return [list(S) for S in product((0, 1), repeat=len(I))
            if consistent(S, I, beta, p, theta0, d, TR, R)]


def phi(S):
    """Latent spike timing of Proposition 2: phi(S)[t] = sum_{k<=t} S[k] (t - k + 1)."""
    out = []
    for t in range(1, len(S) + 1):
        out.append(sum(S[k - 1] * (t - k + 1) for k in range(1, t + 1)))
    return out
