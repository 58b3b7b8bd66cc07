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


def test_project_backward_matches_loops_and_adjoint():
    """grad_W, grad_bias, grad_S are the adjoint of I = W S + b: explicit loops on a tiny case,
    and <W S + b, gI> = <W, gW> + <b, gb>, <W S', gI> = <S', gS> for any real S'."""
    rng = np.random.default_rng(3)
    B, Nin, N, T = 2, 5, 4, 7
    W = rng.standard_normal((N, Nin)).astype(np.float32)
    S = rng.random((B, Nin, T)) < 0.4
    b = rng.standard_normal(N).astype(np.float32)
    gI = rng.standard_normal((B, N, T))
    gW, gS, gb = project.project_backward(W, S, gI)
    for i in range(N):
        for j in range(Nin):
            acc = sum(gI[bb, i, t] for bb in range(B) for t in range(T) if S[bb, j, t])
            assert abs(gW[i, j] - acc) < 1e-12
        assert abs(gb[i] - gI[:, i, :].sum()) < 1e-12
    lhs = float((project.project(W, S, b) * gI).sum())
    rhs = float((W.astype(np.float64) * gW).sum() + (b.astype(np.float64) * gb).sum())
    assert abs(lhs - rhs) < 1e-10 * max(1.0, abs(lhs))
    Sr = rng.standard_normal((B, Nin, T))
    lhs = float((np.einsum("ij,bjt->bit", W.astype(np.float64), Sr) * gI).sum())
    assert abs(lhs - float((Sr * gS).sum())) < 1e-10 * max(1.0, abs(lhs))
