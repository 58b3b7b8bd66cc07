"""The torch.autograd.Function wrapper: forward = block forward, backward = block backward,
gradients reaching the current and the per-neuron parameters as the oracle's BPTT says."""
import numpy as np
import pytest
import torch

from oracle import ref
from paper_2311_11390_gb300 import synth
from tests import parity

pytestmark = pytest.mark.gpu
cuda = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")


@cuda
@pytest.mark.parametrize("attached", [False, True])
def test_autograd_function_matches_oracle_bptt(attached):
    from paper_2311_11390_gb300 import autograd as ag
    w = synth.population(seed=2, B=3, N=48, T=900, tau_adapt=(80.0, 300.0), d=(0.05, 0.4))
    I = torch.from_numpy(w.I).cuda().requires_grad_(True)
    P = {k: torch.from_numpy(np.asarray(getattr(w.params, k))).cuda().requires_grad_(True)
         for k in ("tau_mem", "tau_adapt", "theta0", "d", "R")}
    S = ag.alif_spikes(I, P["tau_mem"], P["tau_adapt"], P["theta0"], P["d"], P["R"], dt=w.dt, arp=w.arp,
                       attached=attached)
    rng = np.random.default_rng(0)
    gS = rng.standard_normal(w.I.shape).astype(np.float32)
    (S * torch.from_numpy(gS).cuda()).sum().backward()
    res = parity.compare_forward(S.detach().cpu().numpy().astype(np.uint8), None, None, w.I, w.params, w.dt, w.arp)
    parity.assert_forward_parity(res)
    ob = ref.backward(w.I, parity.oracle_params(w.params), w.dt, w.arp, gS.astype(np.float64), force=res["force"],
                      attached=attached)
    at = parity.GRAD_ATOL_FRAC_COUPLED if attached else parity.GRAD_ATOL_FRAC
    parity.grad_close(I.grad.cpu().numpy(), ob.gI, what="grad_I", atol_frac=at)
    for k, n in (("tau_mem", "g_tau_mem"), ("tau_adapt", "g_tau_adapt"), ("theta0", "g_theta0"), ("d", "g_d"),
                 ("R", "g_R")):
        parity.grad_close(P[k].grad.cpu().numpy(), getattr(ob, n).sum(0), what=n, atol_frac=at)


@cuda
def test_layer_module_trains_parameters():
    from paper_2311_11390_gb300 import autograd as ag
    layer = ag.ALIFLayer(16, dt=1.0, arp=2.0).cuda()
    I = (1.5 + 0.5 * torch.randn(2, 16, 300, device="cuda")).requires_grad_(True)
    S = layer(I)
    S.sum().backward()
    for p in layer.parameters():
        assert p.grad is not None and torch.isfinite(p.grad).all()
    assert I.grad is not None and I.grad.abs().sum() > 0
