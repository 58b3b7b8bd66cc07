"""CPU checks of the C ABI: the library builds, loads without a GPU, exports every
function include/alif.h declares, and its host-only calls validate arguments."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"^\s*(?:int|int64_t|size_t|void)\s+\**(\w+)\s*\(", text, re.M))
    return names


@pytest.fixture(scope="module")
def L():
    from paper_2311_11390_gb300 import alif
    return alif.lib()


def test_exports_every_declared_symbol(L):
    names = _declared()
    assert {"alif_forward", "alif_backward", "alif_prepare", "alif_forward_seq"} <= names
    for n in sorted(names):
        assert hasattr(L, n), f"{n} declared in include/ but not exported"


def test_tr_and_prepare_validation():
    from paper_2311_11390_gb300 import alif
    assert alif.tr(0.1, 2.0) == 20
    assert alif.tr(0.05, 2.0) == 40
    assert alif.tr(1.0, 2.0) == 2
    for bad in [(0.3, 1.0), (0.0, 1.0), (0.1, -1.0), (0.1, 0.05), (float("nan"), 1.0)]:
        with pytest.raises(alif.AlifError):
            alif.tr(*bad)
    ok = dict(tau_mem=[20.0], tau_adapt=[200.0], theta0=[1.0], d=[0.1], R=[1.0])
    tab = alif.prepare(**ok, dt_ms=0.1, arp_ms=2.0)
    beta = np.exp(-0.1 / 20.0)
    assert abs(float(tab[0, 0]) + float(tab[0, 1]) - beta) < 1e-15
    assert tab.view(np.int32)[0, 13] == 20 and tab.view(np.int32)[0, 14] == 20
    for key, val in [("tau_mem", [0.0]), ("tau_adapt", [-1.0]), ("theta0", [0.0]), ("d", [-0.1]),
                     ("R", [float("inf")])]:
        with pytest.raises(alif.AlifError):
            alif.prepare(**{**ok, key: val}, dt_ms=0.1, arp_ms=2.0)
    t1 = alif.prepare(**ok, dt_ms=0.1, arp_ms=0.1)
    assert t1.view(np.int32)[0, 13] == 1 and t1.view(np.int32)[0, 14] == 2


def test_ckpt_count(L):
    from paper_2311_11390_gb300 import alif
    assert [alif.ckpt_count(t) for t in (0, 1, 256, 257, 1000)] == [0, 1, 1, 2, 4]


def test_last_error_is_thread_local_message(L):
    from paper_2311_11390_gb300 import alif
    with pytest.raises(alif.AlifError) as e:
        alif.tr(0.3, 1.0)
    assert "not an integer" in str(e.value)


def test_recurrent_host_validation(L):
    """alif_forward_recurrent / alif_delay_spikes reject bad arguments on the host, before
    any device work: unsupported N or T_R, a non-integer ARP/DT, missing arrays, a negative
    delay, an aliased delayed raster."""
    c = ctypes.c_void_p
    fake = c(16)  # never dereferenced: every call below fails validation first
    rc = L.alif_forward_recurrent(1, 9000, 100, fake, fake, fake, 0.1, 2.0, None, None, fake, None, None, None)
    assert rc == -4                                      # ALIF_EUNSUPPORTED: N > 8192
    rc = L.alif_forward_recurrent(1, 64, 100, fake, fake, fake, 0.1, 200.0, None, None, fake, None, None, None)
    assert rc == -4                                      # T_R = 2000 > 1023
    rc = L.alif_forward_recurrent(1, 64, 100, fake, fake, fake, 0.3, 1.0, None, None, fake, None, None, None)
    assert rc == -2                                      # ALIF_ETR
    rc = L.alif_forward_recurrent(1, 64, 100, None, fake, fake, 0.1, 2.0, None, None, fake, None, None, None)
    assert rc == -1                                      # I_ff missing
    assert L.alif_delay_spikes(1, 4, 100, -1, fake, c(32), None) == -1
    assert L.alif_delay_spikes(1, 4, 100, 3, fake, fake, None) == -1
    assert L.alif_forward_recurrent(0, 64, 100, None, None, None, 0.1, 2.0, None, None, None, None, None, None) == 0


def test_readout_weights_host(L):
    """The readout's time weights w_t = 1 - beta_o^(T-t) (host, FP64 rounded once) and their sum;
    invalid arguments are refused."""
    from paper_2311_11390_gb300 import alif
    T, dt, tau = 777, 1.0, 20.0
    w, s = alif.readout_weights(T, dt, tau, "cpu")
    beta = np.exp(-dt / tau)
    ref = 1.0 - beta ** (T - np.arange(T, dtype=np.float64))
    assert np.array_equal(w.numpy(), ref.astype(np.float32))
    assert abs(s - ref.sum()) <= 1e-9 * ref.sum()
    assert L.alif_readout_weights(10, -1.0, 20.0, None, None) == -1
    assert L.alif_readout_weights(-1, 1.0, 20.0, None, None) == -3


def test_fused_forward_host_validation(L):
    """alif_forward_fused refuses unsupported widths, bad capacities and misaligned arrays on
    the host, before any device work."""
    c = ctypes.c_void_p
    ok = c(1 << 20)
    args = lambda Nin, cap, I: (1, Nin, 8, 64, ok, ok, None, ok, None, cap, I, ok, None, None, ok, 1 << 30, None)
    assert L.alif_forward_fused(*args(2000, 64, ok)) == -4       # Nin > 1024
    assert L.alif_forward_fused(*args(100, 0, ok)) == -1         # no bucket capacity
    assert L.alif_forward_fused(*args(100, 64, c((1 << 20) + 4))) == -3  # I not 16-byte aligned


def test_layout_setting_host(L):
    """The forward layout setting returns the previous setting, takes 0 / 1 / 2 and refuses
    anything else without changing the setting."""
    prev = L.alif_forward_layout(0)
    try:
        assert L.alif_forward_layout(2) == 0
        assert L.alif_forward_layout(1) == 2
        assert L.alif_forward_layout(3) == -1
        assert L.alif_forward_layout(-1) == -1
        assert L.alif_forward_layout(0) == 1
    finally:
        L.alif_forward_layout(prev)


@pytest.mark.parametrize("name", ["alif_backward_window", "alif_forward_window"])
def test_window_settings_host(L, name):
    """The window-length settings return the previous setting, take 0 / 256 / 512 and refuse
    anything else without changing the setting."""
    fn = getattr(L, name)
    prev = fn(0)
    try:
        assert fn(256) == 0
        assert fn(512) == 256
        assert fn(100) == -1
        assert fn(0) == 512
    finally:
        fn(prev)
