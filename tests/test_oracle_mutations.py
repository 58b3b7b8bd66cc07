"""Plant plausible mistakes in a copy of the oracle and check that the pins catch them.

Each mutant is the oracle's C source with one small edit (a flipped comparison,
an off-by-one in the refractory counter, a dropped reset, a wrong adaptation
index, a dropped surrogate term ...).  It is compiled on the CPU into a
temporary library and run through the pin tests; every mutant must fail at
least one of them.  Nothing here runs on a GPU.
"""
import ctypes
import os
import subprocess
import tempfile

import pytest

from oracle import ref
import tests.test_oracle_pins as pins
import tests.test_oracle_recurrent as rpins

MUTANTS = {
    "strict_gt_to_ge": ("int s = (V_t > theta);\n        if (force", "int s = (V_t >= theta);\n        if (force"),
    "rec_strict_gt_to_ge": ("int s = (V_t > theta);                                     /* Eq 1 */",
                            "int s = (V_t >= theta);                                    /* Eq 1 */"),
    "arp_ge_to_gt": ("int admit = (C >= j->TR);", "int admit = (C > j->TR);"),
    "drop_reset": ("* (1.0 - S_prev);", ";"),
    "adapt_uses_current_spike": ("double a_t = p * a_prev + S_prev;", "double a_t = p * a_prev;"),
    "theta_sign": ("double theta = th0 + d * a_t;", "double theta = th0 - d * a_t;"),
    "leak_factor": ("(1.0 - beta) * R * Iin) * (1.0 - S_prev)", "R * Iin) * (1.0 - S_prev)"),
    "surrogate_slope": ("const double den = slope * fabs(u) + 1.0;",
                        "const double den = slope * u + 1.0;"),
    "mg_side_sign": ("- 0.15 * normal_density(u, -3.0, 3.0);", "+ 0.15 * normal_density(u, -3.0, 3.0);"),
    "boxcar_width": ("return fabs(u) <= 0.5 ? 0.5 : 0.0;", "return fabs(u) <= 0.25 ? 0.5 : 0.0;"),
    "gI_reset_factor": ("(m[k] ? 1.0 : 0.0) * (1.0 - s_km1) * GV;", "(m[k] ? 1.0 : 0.0) * GV;"),
    "gV_reset": ("beta * (1.0 - s_k) * GV_next", "beta * GV_next"),
    "attached_a_path": ("GS += Ga_next - Vpre_next * GV_next;", "GS += -Vpre_next * GV_next;"),
    "attached_input_term": ("const double Vpre_next = beta * V[k] + (1.0 - beta) * R * Iin_next;",
                            "const double Vpre_next = beta * V[k];"),
    "rec_delay": ("if (k >= TR)\n                for (int64_t jn = 0; jn < N; ++jn)\n"
                  "                    if (Sb[jn * T + (k - TR)]) pre[npre++] = jn;",
                  "if (k >= TR + 1)\n                for (int64_t jn = 0; jn < N; ++jn)\n"
                  "                    if (Sb[jn * T + (k - TR - 1)]) pre[npre++] = jn;"),
    "rec_sign": ("Irec += (double)j->W_rec[i * N + pre[q]];", "Irec -= (double)j->W_rec[i * N + pre[q]];"),
    "rec_transposed": ("Irec += (double)j->W_rec[i * N + pre[q]];", "Irec += (double)j->W_rec[pre[q] * N + i];"),
    "g_beta_term": ("g_beta += (1.0 - s_km1) * (V_km1 - R * Iin) * GV;",
                    "g_beta += (1.0 - s_km1) * V_km1 * GV;"),
}


def _build_mutant(name, tmpdir):
    old, new = MUTANTS[name]
    src = open(os.path.join(os.path.dirname(ref.__file__), "alif_oracle.c")).read()
    assert src.count(old) == 1, name
    path = os.path.join(tmpdir, f"{name}.c")
    open(path, "w").write(src.replace(old, new))
    so = os.path.join(tmpdir, f"{name}.so")
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                           "-o", so, path, "-lm", "-lpthread"])
    return so


def _pin_calls():
    """(name, callable(ref_module)) for a fast subset of the pins."""
    calls = []
    for case in pins.LIF_CASES:
        calls.append(("lif", lambda r, c=case: pins.test_lif_first_passage_closed_form(r, *c)))
    calls.append(("filter", pins.test_no_spike_membrane_is_linear_filter))
    calls.append(("tie", pins.test_strict_threshold_at_exact_tie))
    for seed in range(8):
        calls.append(("exact", lambda r, s=seed: pins.test_oracle_matches_exact_rational(r, s)))
    for seed, arp in [(0, 2.0), (3, 0.3)]:
        calls.append(("blocks", lambda r, s=seed, a=arp: pins.test_oracle_equals_paper_blocks(r, s, a)))
    calls.append(("invariants", lambda r: pins.test_arp_invariants(r, 0)))
    for seed, arp in [(0, 1.5), (2, 0.5)]:
        calls.append(("autograd", lambda r, s=seed, a=arp: pins.test_backward_matches_autograd(r, s, a)))
    calls.append(("fd", pins.test_backward_matches_finite_differences))
    for sgt in ("multi_gaussian", "boxcar"):
        calls.append(("surrogates", lambda r, s_=sgt: pins.test_backward_surrogates_match_autograd(r, s_)))
    calls.append(("attached", lambda r: pins.test_backward_attached_matches_autograd(r, "fast_sigmoid", 1.5)))
    calls.append(("rec_ff", lambda r: rpins.test_recurrent_without_weights_is_feedforward(r, 2.0)))
    calls.append(("rec_tie", rpins.test_recurrent_strict_threshold_at_exact_tie))
    calls.append(("rec_delay", lambda r: rpins.test_one_presynaptic_spike_arrives_T_R_later(r, 2.0, 0.1)))
    for seed, arp, scale in [(0, 2.0, 1.5), (3, 0.3, -2.0)]:
        calls.append(("rec_blocks", lambda r, a=(seed, arp, scale): rpins.test_recurrent_oracle_equals_paper_blocks(r, *a)))
    return calls


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, monkeypatch):
    ref._load()
    with tempfile.TemporaryDirectory() as tmp:
        so = _build_mutant(name, tmp)
        lib = ctypes.CDLL(so)
        for fn in ("oracle_tr", "oracle_alif_forward", "oracle_alif_backward", "oracle_alif_forward_recurrent"):
            getattr(lib, fn).argtypes = getattr(ref._lib, fn).argtypes
            getattr(lib, fn).restype = getattr(ref._lib, fn).restype
        monkeypatch.setattr(ref, "_lib", lib)
        caught = []
        for label, call in _pin_calls():
            try:
                call(ref)
            except (AssertionError, ValueError):
                caught.append(label)
        assert caught, f"mutant {name} passed every pin"
