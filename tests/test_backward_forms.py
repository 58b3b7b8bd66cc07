"""The parameter-gradient sums the backward kernel evaluates, checked on the FP64 oracle (no GPU).

With the reset and the ARP mask detached (Supplementary, "Detaching gradients"), Eq 2 gives
dV[t]/dbeta = V[t-1] (1 - S[t-1]) - R m[t] I[t] and dV[t]/dR = (1 - beta) m[t] I[t], while
dL/dI[t] = (1 - beta) R m[t] G_V[t] with G_V the total gradient reaching V[t].  So, per neuron,
    dL/dtau_mem = dbeta/dtau_mem * sum_t (V[t-1] (1 - S[t-1]) - R m[t] I[t]) G_V[t],
    dL/dR       = sum_t dL/dI[t] I[t] / R.
The kernel takes the beta sum in its same-step form: V[t] - (1 - beta) R m[t] I[t] is beta times
the membrane entering step t, and (1 - beta) R + beta R = R, so
    sum_t (V[t-1] (1 - S[t-1]) - R m I[t]) G_V[t] = (1 / beta) sum_t (V[t] - R m I[t]) G_V[t].
Here both forms are built from the oracle's forward traces and its dL/dI, and compared with each
other and with the oracle BPTT's own dL/dtau_mem and dL/dR.  G_V is recovered from dL/dI on the
admitted steps only; on the others every term is 0 (the membrane entering a masked step is 0), so
the reset factor itself is not probed here, but the gain (R, not c) of the input term, the 1/beta of
the same-step form (dropping it is off by 5 %), the sign and the step alignment are.
"""
import numpy as np
import pytest

from oracle import ref
from paper_2311_11390_gb300 import synth


@pytest.mark.parametrize("seed, arp, tau_mem", [(0, 2.0, (2.0, 40.0)), (1, 0.3, (0.5, 5.0)), (2, 1.0, (20.0, 200.0))])
def test_beta_sum_forms_and_oracle_adjoint(seed, arp, tau_mem):
    w = synth.population(seed=seed, B=2, N=12, T=3000, dt=0.1, arp=arp, bias=(1.5, 4.0), tau_mem=tau_mem,
                         tau_adapt=(20.0, 400.0), d=(0.0, 0.8))
    P = w.params
    params = ref.Params(P.tau_mem, P.tau_adapt, P.theta0, P.d, P.R)
    o = ref.forward(w.I, params, w.dt, w.arp)
    assert o.S.sum() > 100
    gS = np.random.default_rng(seed).standard_normal(w.I.shape)
    b = ref.backward(w.I, params, w.dt, w.arp, gS)

    tau = P.tau_mem.astype(np.float64)[None, :, None]
    beta = np.exp(-w.dt / tau)
    R = P.R.astype(np.float64)[None, :, None]
    c = (1.0 - beta) * R
    I = w.I.astype(np.float64)
    m = o.mask.astype(np.float64)
    V, S = o.V, o.S.astype(np.float64)
    GV = np.where(m > 0, b.gI / c, 0.0)           # dL/dI = c m G_V; G_V's masked steps meet 0 terms
    Vent = np.zeros_like(V)                       # membrane entering each step (rest at t = 0)
    Vent[..., 1:] = V[..., :-1] * (1.0 - S[..., :-1])
    shifted = ((Vent - R * m * I) * GV).sum(-1)
    same_step = ((V - R * m * I) * GV).sum(-1) / beta[..., 0]
    scale = (np.abs(Vent - R * m * I) * np.abs(GV)).sum(-1) + 1e-300
    assert np.all(np.abs(shifted - same_step) <= 1e-10 * scale)

    dbeta_dtau = (beta * w.dt / tau ** 2)[..., 0]
    np.testing.assert_allclose(dbeta_dtau * shifted, b.g_tau_mem, rtol=1e-9, atol=1e-12 * np.abs(b.g_tau_mem).max())
    gR = (b.gI * I).sum(-1) / R[..., 0]
    np.testing.assert_allclose(gR, b.g_R, rtol=1e-9, atol=1e-12 * np.abs(b.g_R).max())
