"""The CUDA block backward against central finite differences (no oracle BPTT involved).

With the loss on the V and a traces only (dL/dS = 0) no surrogate enters: for fixed
spike times V and a are smooth functions of the input current, R, tau_mem and
tau_adapt, so the exact gradient is the limit of central differences of the forward
model, as long as no spike moves under the perturbation (checked).  The differences are
taken on the plain FP64 step-by-step model (Eqs 1-5), evaluated by the oracle's forward
only; the gradients come from alif_backward on the GPU.  Tolerance: 1e-4 relative, the
gradient tolerance of the method's parity bar.
"""
import numpy as np
import pytest
import torch

from oracle import ref
from tests import parity

pytestmark = pytest.mark.gpu
cuda = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")


def _params(tm, ta, th0, d, R):
    return ref.Params(np.asarray(tm, np.float64), np.asarray(ta, np.float64), np.asarray(th0, np.float64),
                      np.asarray(d, np.float64), np.asarray(R, np.float64))


@cuda
@pytest.mark.parametrize("T, arp", [(700, 2.0), (300, 0.1)])
def test_gpu_backward_matches_central_differences(T, arp):
    from paper_2311_11390_gb300 import alif
    alif.lib()
    rng = np.random.default_rng(T)
    N, dt = 3, 0.1
    I32 = (1.8 + 0.3 * rng.standard_normal((1, N, T))).astype(np.float32)
    tm = np.array([12.0, 25.0, 18.0], np.float32)
    ta = np.array([80.0, 300.0, 150.0], np.float32)
    th0 = np.array([1.0, 0.9, 1.1], np.float32)
    d = np.array([0.2, 0.4, 0.1], np.float32)
    R = np.array([1.1, 0.9, 1.0], np.float32)
    wV = rng.standard_normal((1, N, T)).astype(np.float32)
    wa = rng.standard_normal((1, N, T)).astype(np.float32)

    table = alif.neuron_table(tm, ta, th0, d, R, dt, arp)
    It = torch.from_numpy(I32).cuda()
    out = alif.forward(It, table)
    gI, _, gp = alif.backward(It, table, out["spikes"], torch.zeros_like(It), ckpt=out["ckpt"],
                              grad_v=torch.from_numpy(wV).cuda(), grad_a=torch.from_numpy(wa).cuda())
    torch.cuda.synchronize()
    assert alif.device_status() == 0
    gI, gp = gI.cpu().numpy().astype(np.float64), gp.cpu().numpy().astype(np.float64)

    I64 = I32.astype(np.float64)
    base = ref.forward(I32, _params(tm, ta, th0, d, R), dt, arp)
    S_gpu = alif.unpack_spikes(out["spikes"], T).cpu().numpy()
    assert np.array_equal(S_gpu, base.S) and base.S.sum() >= 4

    def loss(I_, tm_, ta_, R_):
        o = ref.forward(I_.astype(np.float32), _params(tm_, ta_, th0, d, R_), dt, arp)
        assert np.array_equal(o.S, base.S), "a spike moved under the perturbation"
        return float((o.V * wV).sum() + (o.a * wa).sum())

    tm64, ta64, R64 = tm.astype(np.float64), ta.astype(np.float64), R.astype(np.float64)
    for i in range(N):
        for k, name, eps in ((0, "tm", 1e-5), (1, "ta", 1e-4), (4, "R", 1e-6)):
            def f(e):
                x = {"tm": tm64.copy(), "ta": ta64.copy(), "R": R64.copy()}
                x[name][i] += e
                return loss(I64, x["tm"], x["ta"], x["R"])
            num = (f(eps) - f(-eps)) / (2 * eps)
            assert abs(gp[k, i] - num) <= 1e-4 * abs(num) + 1e-9, (name, i, gp[k, i], num)
    # the current (FP32 in the model): perturb by amounts whose sums stay exact in FP32
    for (i, t) in [(0, 5), (0, 250), (1, 80), (2, T - 1), (1, T // 2)]:
        def f(e):
            I2 = I64.copy()
            I2[0, i, t] += e
            return loss(I2, tm64, ta64, R64)
        eps = 2.0 ** -12
        num = (f(eps) - f(-eps)) / (2 * eps)
        assert abs(gI[0, i, t] - num) <= 1e-4 * abs(num) + 1e-7, (i, t, gI[0, i, t], num)
    # no surrogate term in this loss: the threshold gradients vanish
    assert np.all(gp[2] == 0) and np.all(gp[3] == 0)
