"""Writes lif_first_passage.txt from the closed form alone (no simulator is run).

Discrete LIF (Eq 2 with d = 0, constant input I, from rest): V[k] = R I (1 - beta^k) with
beta = exp(-DT/tau), so the first spike is the first k with R I (1 - beta^k) > theta0, i.e.
k* = floor(t*/DT) + 1 with t* = -tau ln(1 - theta0 / (R I)); after a spike the reset zeroes V
and the ARP holds the input off for max(T_R, 2) - 1 steps, so every later interval is
max(T_R, 2) - 1 + k*.  Inputs are float32-rounded currents, as the simulators receive them.
"""
import math
import os

import numpy as np

CASES = [  # tau_mem, dt, theta0, R, I, T_R
    (20.0, 0.1, 1.0, 1.0, 1.37, 20),
    (10.0, 0.1, 1.0, 1.5, 0.9, 10),
    (5.0, 1.0, 0.7, 1.0, 2.3, 2),
    (30.0, 0.05, 1.2, 2.0, 0.77, 40),
    (20.0, 0.1, 1.0, 1.0, 5.0, 1),
    (15.0, 0.1, 0.9, 1.0, 1.05, 20),
]


def main():
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lif_first_passage.txt")
    with open(out, "w") as f:
        f.write("# tau_mem dt theta0 R I(float32) T_R k_star isi   (paper time, first spike at step k_star)\n")
        for tau, dt, th0, R, I, TR in CASES:
            I32 = float(np.float32(I))
            ratio = -tau * math.log(1.0 - th0 / (R * I32)) / dt
            assert abs(ratio - round(ratio)) > 1e-6
            kstar = math.floor(ratio) + 1
            isi = max(TR, 2) - 1 + kstar
            f.write(f"{tau!r} {dt!r} {th0!r} {R!r} {I32!r} {TR} {kstar} {isi}\n")


if __name__ == "__main__":
    main()
