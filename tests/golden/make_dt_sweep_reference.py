"""Writes dt_sweep_reference.txt: the FP64 oracle's spike steps at the fine DT for the first
SAMPLE neurons of the DT-sweep workload (synth.dt_sweep), the reference the speed-accuracy
sweep scores coarser DTs against (the trade-off of the paper's opening figure: simulation
error against DT, here the van Rossum distance to the fine-DT spike train).  Calls only the
oracle and the seeded input generator."""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import ref  # noqa: E402
from paper_2311_11390_gb300 import synth  # noqa: E402

SAMPLE = 32
ARP = 2.0
OUT = os.path.join(HERE, "dt_sweep_reference.txt")


def reference_spikes(sample=SAMPLE, seed=21, n=1024, seconds=1.0):
    w = synth.dt_sweep(seed=seed, n=n, seconds=seconds)
    P = w.params
    params = ref.Params(*(np.asarray(getattr(P, k)[:sample], np.float64)
                          for k in ("tau_mem", "tau_adapt", "theta0", "d", "R")))
    I = np.ascontiguousarray(np.broadcast_to(w.x_fine[None, None, :], (1, sample, w.x_fine.size)))
    o = ref.forward(I, params, w.fine_dt, ARP, records=False)
    return [np.flatnonzero(o.S[0, i]).tolist() for i in range(sample)]


def main():
    spikes = reference_spikes()
    with open(OUT, "w") as f:
        f.write("# DT-sweep reference: synth.dt_sweep(seed=21, n=1024, seconds=1.0), fine DT 0.01 ms, ARP 2 ms;\n")
        f.write("# FP64 oracle (Eqs 1-5) spike steps of neurons 0..%d, one line per neuron: index | steps\n"
                % (SAMPLE - 1))
        for i, s in enumerate(spikes):
            f.write(f"{i} | {' '.join(map(str, s))}\n")


if __name__ == "__main__":
    main()
