"""Golden fixtures: hand-evaluated / closed-form values (tests/golden/) vs the oracle."""
import os

import numpy as np

from oracle import exact, ref

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_phi_fixture():
    """Prop 2's latent timing, evaluated by hand."""
    for line in open(os.path.join(GOLDEN, "phi_prop2.txt")):
        if line.startswith("#") or "|" not in line:
            continue
        s, z = line.split("|")
        assert exact.phi([int(x) for x in s.split()]) == [int(x) for x in z.split()]


def test_lif_first_passage_fixture():
    """First spike and inter-spike interval of the closed form (written by
    make_lif_first_passage.py from the formula alone) reproduced by the FP64 oracle."""
    n = 0
    for line in open(os.path.join(GOLDEN, "lif_first_passage.txt")):
        if line.startswith("#"):
            continue
        tau, dt, th0, R, I, TR, kstar, isi = line.split()
        tau, dt, th0, R, I = map(float, (tau, dt, th0, R, I))
        TR, kstar, isi = int(TR), int(kstar), int(isi)
        assert ref.tr(dt, TR * dt) == TR
        T = kstar + 3 * isi + 1
        out = ref.forward(np.full((1, 1, T), np.float32(I)),
                          ref.Params(np.array([tau]), np.array([100.0]), np.array([th0]), np.array([0.0]),
                                     np.array([R])), dt, TR * dt)
        spikes = (np.flatnonzero(out.S[0, 0]) + 1).tolist()
        assert spikes == [kstar + m * isi for m in range(4)]
        n += 1
    assert n >= 5


def test_dt_sweep_reference_fixture():
    """The DT-sweep reference (written by make_dt_sweep_reference.py from the oracle and the
    seeded inputs) is what the oracle gives now, and it satisfies Eq 4's refractory bound."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("mk_dt", os.path.join(GOLDEN, "make_dt_sweep_reference.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    stored = []
    for line in open(os.path.join(GOLDEN, "dt_sweep_reference.txt")):
        if line.startswith("#"):
            continue
        stored.append([int(x) for x in line.split("|")[1].split()])
    assert stored == mk.reference_spikes()
    TR = ref.tr(0.01, mk.ARP)
    for s in stored:
        assert all(b - a >= TR for a, b in zip(s, s[1:]))
    assert sum(len(s) for s in stored) > 50
