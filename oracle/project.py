"""Synaptic projection oracle -- TEST INFRASTRUCTURE ONLY.

Feedforward input current of Eq 3 (Section 2) and Proposition 3:
    I[b, i, t] = bias_i + sum_j W[i, j] * S_in[b, j, t]
computed in float64 from the exact float32 values of W (a library matmul is the
only step).  Also the definition of the split of an FP32 weight into two BF16
terms, hi = bf16(W) and lo = bf16(W - hi), both with IEEE round-to-nearest-even,
written out on the float32 bit pattern.
"""
from __future__ import annotations

import numpy as np


def project(W: np.ndarray, S_in: np.ndarray, bias: np.ndarray | None = None) -> np.ndarray:
    """W: [N, Nin] float32; S_in: [B, Nin, T] in {0,1}; bias: [N] or None -> [B, N, T] float64."""
    W64 = np.asarray(W, dtype=np.float32).astype(np.float64)
    S64 = np.asarray(S_in).astype(np.float64)
    out = np.einsum("ij,bjt->bit", W64, S64, optimize=True)
    if bias is not None:
        out += np.asarray(bias, dtype=np.float32).astype(np.float64)[None, :, None]
    return out


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (nearest, ties to even); returned as float32.
    NaN/Inf are passed through (NaN kept quiet)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    rounded = (u + 0x7FFF + lsb) >> 16
    out = (rounded << 16).astype(np.uint32)
    nonfinite = ~np.isfinite(x)
    out[nonfinite] = (u[nonfinite].astype(np.uint32) & 0xFFFF0000) | np.where(
        np.isnan(x[nonfinite]), 0x00400000, 0).astype(np.uint32)
    return out.view(np.float32)


def bf16_bits(x: np.ndarray) -> np.ndarray:
    """uint16 bit patterns of bf16_round(x)."""
    return (bf16_round(x).view(np.uint32) >> 16).astype(np.uint16)


def split_bf16(W: np.ndarray):
    """(hi, lo) as float32 arrays holding bf16 values: hi = bf16(W), lo = bf16(W - hi)."""
    W = np.ascontiguousarray(W, dtype=np.float32)
    hi = bf16_round(W)
    lo = bf16_round((W.astype(np.float64) - hi.astype(np.float64)).astype(np.float32))
    return hi, lo


def project_backward(W: np.ndarray, S_in: np.ndarray, grad_I: np.ndarray):
    """Adjoint of `project` in float64: grad_W[i,j] = sum_{b,t} gI[b,i,t] S[b,j,t],
    grad_bias[i] = sum_{b,t} gI[b,i,t], grad_S[b,j,t] = sum_i W[i,j] gI[b,i,t]."""
    g = np.asarray(grad_I, dtype=np.float64)
    S64 = np.asarray(S_in).astype(np.float64)
    W64 = np.asarray(W, dtype=np.float32).astype(np.float64)
    gW = np.einsum("bit,bjt->ij", g, S64, optimize=True)
    gb = g.sum(axis=(0, 2))
    gS = np.einsum("ij,bit->bjt", W64, g, optimize=True)
    return gW, gS, gb
