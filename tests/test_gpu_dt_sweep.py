"""Speed-accuracy over DT against the oracle (the trade-off of the paper's opening figure),
at a reduced size: one Ornstein-Uhlenbeck current on a 0.01 ms grid drives fit-like neurons;
each coarser DT sees the current averaged over its bins.  The GPU's fine-DT run equals the
FP64 oracle's, the library's van Rossum distance equals the oracle's on the same trains, and
the distance to the fine-DT oracle reference grows as DT coarsens."""
import numpy as np
import pytest
import torch

from oracle import ref
from oracle import vanrossum as vr
from paper_2311_11390_gb300 import synth
from tests import parity

pytestmark = pytest.mark.gpu
cuda = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")


@cuda
def test_dt_sweep_against_oracle_reference():
    from paper_2311_11390_gb300 import alif
    alif.lib()
    w = synth.dt_sweep(seed=21, n=48, seconds=0.3)
    p, fine, Tf = w.params, w.fine_dt, w.x_fine.size
    n = p.N
    I_fine = np.ascontiguousarray(np.broadcast_to(w.x_fine[None, None, :], (1, n, Tf)))
    o = ref.forward(I_fine, parity.oracle_params(p), fine, 2.0, records=False)
    assert o.S.sum() > 30
    ref_words = torch.from_numpy(synth.pack_bits(o.S[0]).view(np.int32)).cuda()
    dist = {}
    for dt in (0.01, 0.1, 1.0):
        f = int(round(dt / fine))
        x = synth.bin_current(w.x_fine, f)
        I = np.ascontiguousarray(np.broadcast_to(x[None, None, :], (1, n, x.size)))
        table = alif.neuron_table(p.tau_mem, p.tau_adapt, p.theta0, p.d, p.R, dt, 2.0)
        out = alif.forward(torch.from_numpy(I).cuda(), table, want_ckpt=False)
        torch.cuda.synchronize()
        S = alif.unpack_spikes(out["spikes"], x.size).cpu().numpy()
        if dt == 0.01:  # the fine run itself: spike parity with the oracle
            res = parity.compare_forward(S, None, None, I, p, dt, 2.0)
            parity.assert_forward_parity(res)
        placed = synth.place_on_fine_grid(S[0], f)
        words = torch.from_numpy(synth.pack_bits(placed).view(np.int32)).cuda()
        loss = torch.empty(n, device="cuda")
        alif.vanrossum_forward(words, ref_words, Tf, fine, 5.0, 256 * ((Tf + 255) // 256), loss=loss)
        lo = loss.cpu().numpy()
        ol, _ = vr.forward(placed, o.S[0], fine, 5.0)
        np.testing.assert_allclose(lo, ol, rtol=1e-4, atol=1e-6)
        dist[dt] = float(lo.mean())
    assert dist[0.01] <= 1e-6
    assert dist[1.0] > dist[0.1] > dist[0.01]
