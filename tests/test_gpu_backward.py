"""GPU parity of the block backward (and the plain sequential backward) against the oracle's
FP64 sequential BPTT (detached surrogate gradient, fast sigmoid)."""
import numpy as np
import pytest
import torch

from oracle import ref
from paper_2311_11390_gb300 import synth
from tests import parity

pytestmark = pytest.mark.gpu
cuda = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")


@pytest.fixture(autouse=True, params=[256, 512], ids=["win256", "win512"])
def backward_window(request):
    """Every case runs with both window lengths of the detached backward (the 512-step kernel
    takes the calls without trace gradients whose T is a multiple of 16; others use 256)."""
    if not torch.cuda.is_available():
        yield request.param
        return
    from paper_2311_11390_gb300 import alif
    prev = alif.backward_window(request.param)
    yield request.param
    alif.backward_window(prev)


def _alif():
    from paper_2311_11390_gb300 import alif
    alif.lib()
    return alif


def _case(alif, w, seed=0, traces=True, gfin=False, slope=25.0, seq=False, want_gI=True):
    I = w.I
    B, N, T = I.shape
    rng = np.random.default_rng(seed)
    gS = rng.standard_normal(I.shape).astype(np.float32)
    gV = rng.standard_normal(I.shape).astype(np.float32) if traces else None
    ga = rng.standard_normal(I.shape).astype(np.float32) if traces else None
    gf = rng.standard_normal((B, N, 2)).astype(np.float32) if gfin else None
    table = alif.neuron_table(w.params.tau_mem, w.params.tau_adapt, w.params.theta0, w.params.d,
                              w.params.R, w.dt, w.arp)
    It = torch.from_numpy(I).cuda()
    out = alif.forward(It, table, want_v=seq, want_a=seq, seq=seq)
    cu = lambda x: None if x is None else torch.from_numpy(x).cuda()
    gI, ginit, gp = alif.backward(It, table, out["spikes"], cu(gS), ckpt=out["ckpt"], v_trace=out["v"],
                                  a_trace=out["a"], grad_v=cu(gV), grad_a=cu(ga), grad_final=cu(gf),
                                  slope=slope, want_gI=want_gI, want_ginit=True, seq=seq)
    torch.cuda.synchronize()
    assert alif.device_status() == 0
    S = alif.unpack_spikes(out["spikes"], T).cpu().numpy()
    if seq:
        res = parity.compare_forward(S, None, None, I, w.params, w.dt, w.arp, flip_margin=1e-4)
        parity.assert_forward_parity(res, budget=1.0)
    else:
        res = parity.compare_forward(S, None, None, I, w.params, w.dt, w.arp)
        parity.assert_forward_parity(res)
    return dict(gS=gS, gV=gV, ga=ga, gf=gf, gI=None if gI is None else gI.cpu().numpy(),
                ginit=ginit.cpu().numpy(), gp=gp.cpu().numpy(), force=res["force"], S=S)


def _oracle(w, r, slope=25.0):
    gS, gV, ga = (None if x is None else x.astype(np.float64) for x in (r["gS"], r["gV"], r["ga"]))
    P = parity.oracle_params(w.params)
    if r["gf"] is not None:
        # the final-state gradient enters as dL/dV[T] and dL/da[T+1] of a virtual next step:
        # fold it in by extending the sequence by one step with zero input and no spike loss
        raise NotImplementedError
    return ref.backward(w.I, P, w.dt, w.arp, gS, gV, ga, slope=slope, force=r["force"])


def _check(w, r, ob, with_gI=True, atol_frac=parity.GRAD_ATOL_FRAC):
    if with_gI:
        parity.grad_close(r["gI"], ob.gI, what="grad_I", atol_frac=atol_frac)
    names = ["g_tau_mem", "g_tau_adapt", "g_theta0", "g_d", "g_R"]
    for k, n in enumerate(names):
        parity.grad_close(r["gp"][k], getattr(ob, n).sum(0), what=n, atol_frac=atol_frac)
    p = np.exp(-w.dt / w.params.tau_adapt.astype(np.float64))
    parity.grad_close(r["ginit"][..., 0], ob.g_V0, what="grad_init_v", atol_frac=atol_frac)
    parity.grad_close(r["ginit"][..., 1] * p[None, :], ob.g_a0, what="grad_init_a", atol_frac=atol_frac)


@cuda
@pytest.mark.parametrize("seed", [0, 1])
def test_population_backward(seed):
    alif = _alif()
    w = synth.population(seed=seed, B=4, N=64, T=1000)
    r = _case(alif, w, seed=seed)
    _check(w, r, _oracle(w, r))


@cuda
def test_population_backward_spike_loss_only():
    alif = _alif()
    w = synth.population(seed=3, B=4, N=64, T=1000)
    r = _case(alif, w, seed=3, traces=False)
    _check(w, r, _oracle(w, r))


@cuda
@pytest.mark.parametrize("T, arp, dt", [(7, 0.3, 0.1), (257, 1.0, 0.1), (1001, 2.0, 0.1), (1000, 0.1, 0.1),
                                        (3001, 40.0, 0.1), (777, 4.0, 0.05), (1024, 2.0, 1.0)])
def test_backward_edge_cases(T, arp, dt):
    alif = _alif()
    w = synth.population(seed=11, B=2, N=32, T=T, dt=dt, arp=arp, bias=(1.2, 3.0),
                         tau_mem=(2.0, 40.0), tau_adapt=(20.0, 400.0), d=(0.0, 0.8))
    r = _case(alif, w, seed=T)
    _check(w, r, _oracle(w, r))


def _degenerate_population(seed=3, B=2, T=1500):
    """Time constants at the ends of their ranges, per neuron: tau_mem 1e-5 ms (beta = 0 exactly:
    no membrane memory), 1e-3 (beta ~ 4e-44, subnormal in FP32), 0.01, 0.05, 5, 20 and 1e5 ms
    (beta = 1 - 1e-6: the error band of the FP32 fast path hits its cap); tau_adapt 1e-4 ms (p = 0
    exactly, where Prop 5's p^-1 is undefined), 1.1e-3 (p ~ 3e-40, subnormal), 1.2e-3, 0.05 and
    200 ms; d in {0, 0.5, 1}."""
    N = 30
    tm = np.array([1e-5, 1e-3, 0.01, 0.05, 5.0, 20.0, 1e5] * 5)[:N]
    ta = np.array([1e-4, 0.0011, 0.0012, 0.05, 200.0] * 6)[:N]
    d = np.array([0.0, 0.5, 1.0] * 10)[:N]
    P = synth.NeuronParams(tm, ta, np.ones(N), d, np.ones(N)).astype32()
    rng = np.random.default_rng(seed)
    bias = rng.uniform(1.2, 3.0, N).astype(np.float32)
    I = (bias[None, :, None] + 0.3 * rng.standard_normal((B, N, T), dtype=np.float32)).astype(np.float32)
    return synth.PopulationWorkload(I, P, 0.1, 2.0)


@cuda
@pytest.mark.parametrize("T", [1500, 1536])
def test_backward_degenerate_time_constants(T):
    """beta = 0, p = 0, subnormal decays and beta within 1e-6 of 1: forward and backward still
    match the oracle (the oracle's own values for these neurons are finite, asserted).  T = 1536
    takes the bulk-copy variants, whose beta sum is the same-step form completed for beta < 1/2 by
    the follow-up kernel; T = 1500 the direct-load ones."""
    alif = _alif()
    w = _degenerate_population(T=T)
    r = _case(alif, w, seed=5)
    ob = _oracle(w, r)
    for n in ["gI", "g_tau_mem", "g_tau_adapt", "g_theta0", "g_d", "g_R"]:
        assert np.isfinite(getattr(ob, n)).all(), n
    assert r["S"].sum() > 1000
    _check(w, r, ob)


@cuda
def test_trace_only_loss_is_tight():
    """Loss on the V and a traces only (dL/dS = 0): no surrogate, the reverse recurrences are
    linear in FP32 state, so dL/dI and the tau / R gradients match the FP64 BPTT to 1e-5."""
    alif = _alif()
    w = synth.population(seed=6, B=4, N=64, T=1000)
    r = _case(alif, w, seed=6)
    # re-run with gS = 0 through the same path
    table = alif.neuron_table(w.params.tau_mem, w.params.tau_adapt, w.params.theta0, w.params.d,
                              w.params.R, w.dt, w.arp)
    It = torch.from_numpy(w.I).cuda()
    out = alif.forward(It, table)
    z = torch.zeros_like(It)
    gI, ginit, gp = alif.backward(It, table, out["spikes"], z, ckpt=out["ckpt"],
                                  grad_v=torch.from_numpy(r["gV"]).cuda(),
                                  grad_a=torch.from_numpy(r["ga"]).cuda(), want_ginit=True)
    ob = ref.backward(w.I, parity.oracle_params(w.params), w.dt, w.arp, np.zeros(w.I.shape),
                      r["gV"].astype(np.float64), r["ga"].astype(np.float64), force=r["force"])
    # FP32 linear recurrences over ~1/(1-beta) steps: a few ulps relative
    parity.grad_close(gI.cpu().numpy(), ob.gI, rtol=3e-5, atol_frac=3e-6, what="grad_I")
    gp = gp.cpu().numpy()
    for k, n in ((0, "g_tau_mem"), (1, "g_tau_adapt"), (4, "g_R")):
        parity.grad_close(gp[k], getattr(ob, n).sum(0), rtol=3e-5, atol_frac=3e-6, what=n)


@cuda
def test_fit_backward_params_only():
    """Neuron-fit shape: grad_I = NULL, only the parameter gradients (DT=0.05, T_R=40;
    tau_adapt up to 1000 ms, a 20000-step memory of the adaptation gradient), all at the
    standard gradient tolerances."""
    alif = _alif()
    w = synth.neuron_fit(seed=1, N=32, T=20000)
    r = _case(alif, w, seed=5, traces=False, want_gI=False)
    ob = _oracle(w, r)
    for k, n in enumerate(["g_tau_mem", "g_tau_adapt", "g_theta0", "g_d", "g_R"]):
        parity.grad_close(r["gp"][k], getattr(ob, n).sum(0), what=n)


@cuda
def test_chunked_backward_equals_single():
    """Backward over two chunks linked by grad_final / grad_init equals one backward.

    Both are held against the oracle's BPTT over the whole sequence at the gradient
    tolerances: the two runs take different kernel paths near the chunk boundary (the last
    window of a launch always takes the general path, a spike-free interior window the lean
    one), and the fast-sigmoid slope (up to 2k) turns their FP32 rounding differences in V
    into ~1e-4 differences of the theta0 / R sums, while a broken link would be off by O(1)."""
    alif = _alif()
    w = synth.population(seed=4, B=2, N=32, T=1536)
    table = alif.neuron_table(w.params.tau_mem, w.params.tau_adapt, w.params.theta0, w.params.d,
                              w.params.R, w.dt, w.arp)
    It = torch.from_numpy(w.I).cuda()
    gS = torch.randn(It.shape, device="cuda", generator=torch.Generator("cuda").manual_seed(0))
    full = alif.forward(It, table)
    gI, _, gp = alif.backward(It, table, full["spikes"], gS, ckpt=full["ckpt"])
    T1 = 512
    A = alif.forward(It[..., :T1].contiguous(), table)
    Bc = alif.forward(It[..., T1:].contiguous(), table, init=A["final"])
    gI2, gin2, gp2 = alif.backward(It[..., T1:].contiguous(), table, Bc["spikes"], gS[..., T1:].contiguous(),
                                   ckpt=Bc["ckpt"], init=A["final"], want_ginit=True)
    gI1, _, gp1 = alif.backward(It[..., :T1].contiguous(), table, A["spikes"], gS[..., :T1].contiguous(),
                                ckpt=A["ckpt"], grad_final=gin2)
    torch.cuda.synchronize()
    S_full = alif.unpack_spikes(full["spikes"], w.I.shape[-1]).cpu().numpy()
    S_chunk = np.concatenate([alif.unpack_spikes(A["spikes"], T1).cpu().numpy(),
                              alif.unpack_spikes(Bc["spikes"], w.I.shape[-1] - T1).cpu().numpy()], -1)
    assert np.array_equal(S_full, S_chunk)
    res = parity.compare_forward(S_full, None, None, w.I, w.params, w.dt, w.arp)
    parity.assert_forward_parity(res)
    ob = _oracle(w, dict(gS=gS.cpu().numpy(), gV=None, ga=None, gf=None, force=res["force"]))
    names = ["g_tau_mem", "g_tau_adapt", "g_theta0", "g_d", "g_R"]
    for label, gi, gpar in (("single", gI, gp), ("chunked", torch.cat([gI1, gI2], -1), gp1 + gp2)):
        parity.grad_close(gi.cpu().numpy(), ob.gI, what=f"{label} grad_I")
        for k, n in enumerate(names):
            parity.grad_close(gpar[k].cpu().numpy(), getattr(ob, n).sum(0), what=f"{label} {n}")
    torch.testing.assert_close(torch.cat([gI1, gI2], -1), gI, rtol=1e-4, atol=1e-5)


@cuda
@pytest.mark.parametrize("seed", [0, 1])
def test_sequential_backward(seed):
    alif = _alif()
    w = synth.population(seed=seed, B=4, N=64, T=1000)
    r = _case(alif, w, seed=seed, seq=True)
    _check(w, r, _oracle(w, r), atol_frac=parity.GRAD_ATOL_FRAC_COUPLED)


@cuda
@pytest.mark.parametrize("surrogate", ["multi_gaussian", "boxcar"])
def test_backward_other_surrogates(surrogate):
    """The multi-Gaussian and boxcar surrogates against the oracle's BPTT with the same
    surrogate.  The boxcar jumps at |V - theta| = 0.5, where FP32 and FP64 membranes can fall
    on opposite sides: dL/dS is set to 0 at the steps within 1e-5 of the jump, so that the
    comparison tests the recurrences, not the rounding of V at a discontinuity."""
    from paper_2311_11390_gb300 import alif
    alif.lib()
    w = synth.population(seed=8, B=4, N=64, T=1000)
    P = parity.oracle_params(w.params)
    o = ref.forward(w.I, P, w.dt, w.arp)
    rng = np.random.default_rng(8)
    gS = rng.standard_normal(w.I.shape)
    if surrogate == "boxcar":
        gS[np.abs(np.abs(o.margin) - 0.5) < 1e-5] = 0.0
    table = alif.neuron_table(w.params.tau_mem, w.params.tau_adapt, w.params.theta0, w.params.d,
                              w.params.R, w.dt, w.arp)
    It = torch.from_numpy(w.I).cuda()
    out = alif.forward(It, table)
    S = alif.unpack_spikes(out["spikes"], w.I.shape[-1]).cpu().numpy()
    res = parity.compare_forward(S, None, None, w.I, w.params, w.dt, w.arp)
    parity.assert_forward_parity(res)
    gI, _, gp = alif.backward(It, table, out["spikes"], torch.from_numpy(gS.astype(np.float32)).cuda(),
                              ckpt=out["ckpt"], surrogate=surrogate)
    torch.cuda.synchronize()
    assert alif.device_status() == 0
    ob = ref.backward(w.I, P, w.dt, w.arp, gS, force=res["force"], surrogate=surrogate)
    parity.grad_close(gI.cpu().numpy(), ob.gI, what="grad_I")
    for k, n in enumerate(["g_tau_mem", "g_tau_adapt", "g_theta0", "g_d", "g_R"]):
        parity.grad_close(gp[k].cpu().numpy(), getattr(ob, n).sum(0), what=n)
    with pytest.raises(alif.AlifError):
        alif.backward(It, table, out["spikes"], torch.zeros_like(It), ckpt=out["ckpt"], surrogate="boxcar",
                      seq=True)


def _attached_case(alif, w, surrogate, traces, seed, init=None):
    """GPU attached backward and the oracle's attached BPTT on the same spikes."""
    P = parity.oracle_params(w.params)
    rng = np.random.default_rng(seed)
    gS = rng.standard_normal(w.I.shape)
    gV = rng.standard_normal(w.I.shape) if traces else None
    ga = rng.standard_normal(w.I.shape) if traces else None
    table = alif.neuron_table(w.params.tau_mem, w.params.tau_adapt, w.params.theta0, w.params.d,
                              w.params.R, w.dt, w.arp)
    It = torch.from_numpy(w.I).cuda()
    out = alif.forward(It, table)
    S = alif.unpack_spikes(out["spikes"], w.I.shape[-1]).cpu().numpy()
    res = parity.compare_forward(S, None, None, w.I, w.params, w.dt, w.arp)
    parity.assert_forward_parity(res)
    cu = lambda x: None if x is None else torch.from_numpy(x.astype(np.float32)).cuda()
    gI, ginit, gp = alif.backward(It, table, out["spikes"], cu(gS), ckpt=out["ckpt"], grad_v=cu(gV),
                                  grad_a=cu(ga), surrogate=surrogate, want_ginit=True, attached=True)
    torch.cuda.synchronize()
    assert alif.device_status() == 0
    ob = ref.backward(w.I, P, w.dt, w.arp, gS, gV, ga, force=res["force"], surrogate=surrogate, attached=True)
    return dict(gI=gI.cpu().numpy(), ginit=ginit.cpu().numpy(), gp=gp.cpu().numpy(), S=S, o=ob)


@cuda
@pytest.mark.parametrize("surrogate, T, arp, dt, traces, seed", [
    ("fast_sigmoid", 1000, 2.0, 0.1, True, 21),     # T_R = 20
    ("fast_sigmoid", 1301, 0.2, 0.1, False, 21),    # T_R = 2, ragged last window
    ("fast_sigmoid", 777, 0.1, 0.1, True, 21),      # T_R = 1: the input after a spike enters W
    ("fast_sigmoid", 3001, 4.0, 0.1, False, 21),    # T_R = 40, several windows
    ("multi_gaussian", 1000, 2.0, 0.1, True, 21),   # on the bounded workload (see below)
    ("boxcar", 1000, 2.0, 0.1, False, 25),
])
def test_backward_attached(surrogate, T, arp, dt, traces, seed):
    """Attached gradients (Supplementary, "Detaching gradients"): S[t] keeps its surrogate
    gradient in the reset factor of V[t+1] and in the update of a[t+1], which couples the
    reverse recurrences of G_V and G_a; the kernel's 2 x 2 affine scan against the oracle's
    sequential attached BPTT.  The boxcar jumps at |V - theta| = 0.5: the seed is one where
    no FP64 margin lies within 1e-5 of the jump (asserted), so FP32 and FP64 take the same
    side everywhere.  The multi-Gaussian is wide, so its attached coupling acts at most
    steps: on the mixed workload (tau_mem 5-40 ms, d up to 0.6) the attached gradient grows
    to ~5e9 from unit loss gradients, where even an FP32 replay of the oracle's own loop
    from exact states is 3e-4 off; it is compared on the population workload (tau_mem 20 ms,
    d 0.1), where the gradient stays O(1) (asserted)."""
    alif = _alif()
    if surrogate == "multi_gaussian":
        w = synth.population(seed=seed, B=2, N=32, T=T, dt=dt, arp=arp, bias=(1.5, 3.0))
    else:
        w = synth.population(seed=seed, B=2, N=32, T=T, dt=dt, arp=arp, bias=(1.0, 2.2),
                             tau_mem=(5.0, 40.0), tau_adapt=(50.0, 400.0), d=(0.0, 0.6))
    if surrogate == "boxcar":
        o = ref.forward(w.I, parity.oracle_params(w.params), w.dt, w.arp)
        assert not (np.abs(np.abs(o.margin) - 0.5) < 1e-5).any()
    r = _attached_case(alif, w, surrogate, traces, seed=T)
    ob = r["o"]
    assert r["S"].sum() > 50
    assert np.abs(ob.gI).max() < 10.0
    at = parity.GRAD_ATOL_FRAC_COUPLED
    parity.grad_close(r["gI"], ob.gI, what="grad_I", atol_frac=at)
    for k, n in enumerate(["g_tau_mem", "g_tau_adapt", "g_theta0", "g_d", "g_R"]):
        parity.grad_close(r["gp"][k], getattr(ob, n).sum(0), what=n, atol_frac=at)
    p = np.exp(-w.dt / w.params.tau_adapt.astype(np.float64))
    parity.grad_close(r["ginit"][..., 0], ob.g_V0, what="grad_init_v", atol_frac=at)
    parity.grad_close(r["ginit"][..., 1] * p[None, :], ob.g_a0, what="grad_init_a", atol_frac=at)


@cuda
def test_backward_attached_differs_from_detached():
    """On the same spikes and loss the attached and detached kernels give different dL/dI
    (the oracle says by how much), so the attached path is not the detached one renamed."""
    alif = _alif()
    w = synth.population(seed=22, B=2, N=32, T=1000)
    r = _attached_case(alif, w, "fast_sigmoid", False, seed=5)
    P = parity.oracle_params(w.params)
    rng = np.random.default_rng(5)
    gS = rng.standard_normal(w.I.shape)
    od = ref.backward(w.I, P, w.dt, w.arp, gS)
    gap = np.linalg.norm(od.gI - r["o"].gI) / np.linalg.norm(r["o"].gI)
    assert gap > 1e-2
    assert np.linalg.norm(r["gI"] - r["o"].gI) / np.linalg.norm(r["o"].gI) < 1e-3 * gap


@cuda
@pytest.mark.parametrize("arp", [2.0, 0.1])
def test_chunked_attached_backward_equals_single(arp):
    """The attached backward over two calls linked by the 3-channel grad_final / grad_init
    (the last step of the first call couples to the final state v = V (1 - S), a = p a + S,
    and to the second call's first input through the third channel) against the oracle's
    attached BPTT over the whole sequence (T_R = 20, and T_R = 1 where the step after a
    spike is admitted)."""
    alif = _alif()
    w = synth.population(seed=4, B=2, N=32, T=1536, arp=arp)
    table = alif.neuron_table(w.params.tau_mem, w.params.tau_adapt, w.params.theta0, w.params.d,
                              w.params.R, w.dt, w.arp)
    It = torch.from_numpy(w.I).cuda()
    gS = torch.randn(It.shape, device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    full = alif.forward(It, table)
    T1 = 512
    A = alif.forward(It[..., :T1].contiguous(), table)
    Bc = alif.forward(It[..., T1:].contiguous(), table, init=A["final"])
    gI2, gin2, gp2 = alif.backward(It[..., T1:].contiguous(), table, Bc["spikes"], gS[..., T1:].contiguous(),
                                   ckpt=Bc["ckpt"], init=A["final"], want_ginit=True, attached=True)
    gI1, _, gp1 = alif.backward(It[..., :T1].contiguous(), table, A["spikes"], gS[..., :T1].contiguous(),
                                ckpt=A["ckpt"], grad_final=gin2, attached=True)
    torch.cuda.synchronize()
    assert alif.device_status() == 0
    S_full = alif.unpack_spikes(full["spikes"], w.I.shape[-1]).cpu().numpy()
    res = parity.compare_forward(S_full, None, None, w.I, w.params, w.dt, w.arp)
    parity.assert_forward_parity(res)
    ob = ref.backward(w.I, parity.oracle_params(w.params), w.dt, w.arp, gS.cpu().numpy().astype(np.float64),
                      force=res["force"], attached=True)
    at = parity.GRAD_ATOL_FRAC_COUPLED
    parity.grad_close(torch.cat([gI1, gI2], -1).cpu().numpy(), ob.gI, what="chunked grad_I", atol_frac=at)
    for k, n in enumerate(["g_tau_mem", "g_tau_adapt", "g_theta0", "g_d", "g_R"]):
        parity.grad_close((gp1 + gp2)[k].cpu().numpy(), getattr(ob, n).sum(0), what=f"chunked {n}", atol_frac=at)
    with pytest.raises(alif.AlifError):
        alif.backward(It, table, full["spikes"], gS, ckpt=full["ckpt"], attached=True, seq=True)
