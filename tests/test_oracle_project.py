"""Pins of the projection oracle (Eq 3 feedforward term) and of the BF16 split definition."""
import numpy as np
import torch

from oracle import project


def test_project_matches_explicit_loops():
    rng = np.random.default_rng(0)
    B, Nin, N, T = 2, 7, 5, 9
    W = rng.standard_normal((N, Nin)).astype(np.float32)
    S = rng.random((B, Nin, T)) < 0.4
    b = rng.standard_normal(N).astype(np.float32)
    out = project.project(W, S, b)
    for bb in range(B):
        for i in range(N):
            for t in range(T):
                acc = float(b[i])
                for j in range(Nin):
                    if S[bb, j, t]:
                        acc += float(W[i, j])
                assert abs(out[bb, i, t] - acc) <= 1e-12 * max(1.0, abs(acc))


def test_bf16_round_matches_torch_conversion():
    """torch's float32 -> bfloat16 cast is IEEE round-to-nearest-even."""
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.standard_normal(100000).astype(np.float32) * 10 ** rng.uniform(-30, 30, 100000).astype(np.float32),
                        np.array([0.0, -0.0, 1.0, 1.00390625, 1.01171875, 3.0e38, 1e-40], np.float32)])
    x = x[np.isfinite(x)]
    mine = project.bf16_round(x)
    theirs = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(mine.view(np.uint32), theirs.view(np.uint32))


def test_split_error_bounds():
    """bf16 keeps 8 significant bits, so round-to-nearest errs by at most 2^-8 relative:
    |W - hi| <= 2^-8 |W| and |W - hi - lo| <= 2^-8 |W - hi| <= 2^-16 |W| (normal range)."""
    rng = np.random.default_rng(2)
    W = (rng.standard_normal(200000) * np.sqrt(2 / 1000)).astype(np.float32)
    hi, lo = project.split_bf16(W)
    W64 = W.astype(np.float64)
    assert np.all(np.abs(W64 - hi) <= 2.0 ** -8 * np.abs(W64))
    assert np.all(np.abs(W64 - hi - lo) <= 2.0 ** -16 * np.abs(W64))
    # exactly representable weights split with lo = 0
    Wx = project.bf16_round(W)
    hx, lx = project.split_bf16(Wx)
    assert np.array_equal(hx, Wx) and np.all(lx == 0)
