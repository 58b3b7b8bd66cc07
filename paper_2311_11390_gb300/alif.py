"""ctypes binding of libalif.so (the C ABI in include/alif.h).

Argument marshalling only: every step of the simulation runs in the CUDA
kernels of the library.  PyTorch supplies device memory and the current
stream.  There is no CPU fallback: if the library cannot be loaded, every
call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import build as _build

ALIF_CKPT_STEPS = 256
NUM_PARAM_GRADS = 5
PARAM_GRAD_NAMES = ("tau_mem", "tau_adapt", "theta0", "d", "R")
NEURON_FLOATS = 16  # sizeof(AlifNeuron) / 4

_lib = None


class AlifError(RuntimeError):
    pass


def lib():
    """Load (building first if needed) the in-tree libalif.so; raises if unavailable."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path) or _build._stale([]):
        try:
            _build.build()
        except Exception as e:  # no toolkit / compile error: fail loudly
            raise AlifError(f"libalif.so is missing and could not be built: {e}") from e
    L = ctypes.CDLL(path)
    P, i64, i32, f32, f64, sz = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_float,
                                 ctypes.c_double, ctypes.c_size_t)
    sig = {
        "alif_last_error": ([P, sz], ctypes.c_int),
        "alif_device_status": ([P, P], ctypes.c_int),
        "alif_forward_stats": ([P, P], ctypes.c_int),
        "alif_tr": ([f64, f64], ctypes.c_int),
        "alif_prepare": ([i64, P, P, P, P, P, f64, f64, P], ctypes.c_int),
        "alif_ckpt_count": ([i64], i64),
        "alif_forward": ([i64, i64, i64, P, P, P, P, P, P, P, P, P], ctypes.c_int),
        "alif_forward_seq": ([i64, i64, i64, P, P, P, P, P, P, P, P], ctypes.c_int),
        "alif_forward_seq_staged": ([i64, i64, i64, P, P, P, P, P, P, P, P], ctypes.c_int),
        "alif_backward_workspace_size": ([i64, i64], sz),
        "alif_backward_window": ([ctypes.c_int], ctypes.c_int),
        "alif_forward_window": ([ctypes.c_int], ctypes.c_int),
        "alif_forward_layout": ([ctypes.c_int], ctypes.c_int),
        "alif_backward_seq": ([i64, i64, i64, P, P, P, P, P, P, P, P, P, P, f32, P, P, P, P, sz, P],
                              ctypes.c_int),
        "syn_split_bf16": ([P, i64, i64, i64, P, P, P], ctypes.c_int),
        "syn_project": ([i64, i64, i64, i64, P, P, i64, P, P, P, P], ctypes.c_int),
        "syn_project_backward_workspace_size": ([i64, i64, i64], sz),
        "syn_project_backward": ([i64, i64, i64, i64, P, P, P, P, P, P, P, sz, P], ctypes.c_int),
        "alif_unpack_spikes": ([i64, i64, P, P, P], ctypes.c_int),
        "alif_vanrossum_forward": ([i64, i64, P, P, f64, f64, i64, P, P, P], ctypes.c_int),
        "alif_pack_spikes": ([i64, i64, P, P, P], ctypes.c_int),
        "syn_transpose_weights": ([P, i64, i64, P, P], ctypes.c_int),
        "syn_project_events": ([i64, i64, i64, i64, P, P, P, P, P], ctypes.c_int),
        "alif_forward_recurrent": ([i64, i64, i64, P, P, P, f64, f64, P, P, P, P, P, P], ctypes.c_int),
        "alif_delay_spikes": ([i64, i64, i64, i64, P, P, P], ctypes.c_int),
        "alif_readout_forward": ([i64, i64, i64, i64, P, P, P, P, f32, P, P, P], ctypes.c_int),
        "alif_readout_backward": ([i64, i64, i64, i64, P, P, f32, P, P, P, P, P, P], ctypes.c_int),
        "alif_cross_entropy": ([i64, i64, P, P, P, P, P, P], ctypes.c_int),
        "alif_vanrossum_backward": ([i64, i64, P, P, f64, f64, i64, i64, P, P, P, P], ctypes.c_int),
        "alif_readout_weights": ([i64, f64, f64, P, P], ctypes.c_int),
        "alif_forward_fused_workspace_size": ([i64, i64, i64, i32], sz),
        "alif_forward_fused": ([i64, i64, i64, i64, P, P, P, P, P, i32, P, P, P, P, P, sz, P], ctypes.c_int),
    }
    optional = {
        "alif_backward_noalloc": ([i64, i64, i64, P, P, P, P, P, P, P, P, P, f32, P, P, P, P], ctypes.c_int),
        "alif_backward_surrogate": ([i64, i64, i64, P, P, P, P, P, P, P, P, P, i32, f32, P, P, P, P, sz, P],
                                    ctypes.c_int),
        "alif_backward_attached": ([i64, i64, i64, P, P, P, P, P, P, P, P, P, P, i32, f32, P, P, P, P, P, sz,
                                    P], ctypes.c_int),
        "alif_backward": ([i64, i64, i64, P, P, P, P, P, P, P, P, P, f32, P, P, P, P, sz, P],
                          ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes, fn.restype = args, res
    for name, (args, res) in optional.items():
        fn = getattr(L, name, None)
        if fn is not None:
            fn.argtypes, fn.restype = args, res
    _lib = L
    return L


def backward_window(steps: int) -> int:
    """Window length of the detached backward: 0 = chosen from B*N, 256 or 512 = forced.
    Returns the previous setting."""
    rc = lib().alif_backward_window(int(steps))
    if rc < 0:
        raise AlifError(f"alif_backward_window({steps}) rejected")
    return rc


def forward_window(steps: int) -> int:
    """Window length of the block forward: 0 = chosen from B*N, 256 or 512 = forced.
    Returns the previous setting."""
    rc = lib().alif_forward_window(int(steps))
    if rc < 0:
        raise AlifError(f"alif_forward_window({steps}) rejected")
    return rc


def forward_layout(layout: int) -> int:
    """Layout of the block forward: 0 = chosen from B*N, 1 = a warp per row, 2 = a lane per row.
    Returns the previous setting."""
    rc = lib().alif_forward_layout(int(layout))
    if rc < 0:
        raise AlifError(f"alif_forward_layout({layout}) rejected")
    return rc


def last_error() -> str:
    buf = ctypes.create_string_buffer(1024)
    lib().alif_last_error(buf, 1024)
    return buf.value.decode(errors="replace")


def _check(rc: int, what: str):
    if rc != 0:
        raise AlifError(f"{what} failed ({rc}): {last_error()}")


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream(device=None):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _f32(t, shape=None):
    if t is None:
        return None
    assert t.dtype == torch.float32 and t.is_contiguous(), "float32 contiguous tensor expected"
    if shape is not None:
        assert tuple(t.shape) == tuple(shape), f"shape {tuple(t.shape)} != {shape}"
    return t


# ------------------------------------------------------------------ host side
def tr(dt_ms: float, arp_ms: float) -> int:
    r = lib().alif_tr(float(dt_ms), float(arp_ms))
    if r < 0:
        raise AlifError(f"alif_tr: {last_error()}")
    return r


def prepare(tau_mem, tau_adapt, theta0, d, R=None, dt_ms: float = 0.1, arp_ms: float = 2.0) -> np.ndarray:
    """FP64 host preparation of the per-neuron constants -> float32 [N, 16] (AlifNeuron rows)."""
    c = lambda x: None if x is None else np.ascontiguousarray(np.asarray(x, dtype=np.float32).reshape(-1))
    tm, ta, th, dd, rr = c(tau_mem), c(tau_adapt), c(theta0), c(d), c(R)
    N = tm.shape[0]
    out = np.zeros((N, NEURON_FLOATS), np.float32)
    p = lambda a: None if a is None else a.ctypes.data_as(ctypes.c_void_p)
    _check(lib().alif_prepare(N, p(tm), p(ta), p(th), p(dd), p(rr), float(dt_ms), float(arp_ms),
                              p(out)), "alif_prepare")
    return out


def neuron_table(tau_mem, tau_adapt, theta0, d, R=None, dt_ms=0.1, arp_ms=2.0, device="cuda") -> torch.Tensor:
    """Prepared constants as a device tensor float32 [N, 16]."""
    return torch.from_numpy(prepare(tau_mem, tau_adapt, theta0, d, R, dt_ms, arp_ms)).to(device)


def ckpt_count(T: int) -> int:
    return int(lib().alif_ckpt_count(int(T)))


def state_tensor(B, N, device="cuda", v=None, a=None, rem=None) -> torch.Tensor:
    """AlifState array [B, N, 3] stored as int32 (v and a are float32 bit patterns)."""
    s = torch.zeros((B, N, 3), dtype=torch.int32, device=device)
    f = s.view(torch.float32)
    if v is not None:
        f[..., 0] = torch.as_tensor(v, dtype=torch.float32, device=device)
    if a is not None:
        f[..., 1] = torch.as_tensor(a, dtype=torch.float32, device=device)
    if rem is not None:
        s[..., 2] = torch.as_tensor(rem, dtype=torch.int32, device=device)
    return s


def state_fields(s: torch.Tensor):
    """(v, a, rem) views of an AlifState tensor."""
    f = s.view(torch.float32)
    return f[..., 0], f[..., 1], s[..., 2]


# --------------------------------------------------------------- forward pass
def forward(I: torch.Tensor, table: torch.Tensor, init: torch.Tensor | None = None, want_v=False,
            want_a=False, want_ckpt=True, want_final=True, seq=False):
    """Block forward (or the plain sequential kernel if seq=True, the staged sequential kernel if
    seq="staged").  I: float32 [B, N, T] on the GPU.  Returns dict(spikes [B,N,ceil(T/32)] int32
    bits, v, a, ckpt, final)."""
    _f32(I)
    B, N, T = I.shape
    dev = I.device
    nwords = (T + 31) // 32
    spikes = torch.empty((B, N, nwords), dtype=torch.int32, device=dev)
    v = torch.empty_like(I) if want_v else None
    a = torch.empty_like(I) if want_a else None
    ckpt = (torch.empty((B, N, max(ckpt_count(T), 1), 3), dtype=torch.int32, device=dev)
            if (want_ckpt and not seq) else None)
    fin = torch.empty((B, N, 3), dtype=torch.int32, device=dev) if want_final else None
    assert table.dtype == torch.float32 and tuple(table.shape) == (N, NEURON_FLOATS)
    if init is not None:
        assert init.dtype == torch.int32 and tuple(init.shape) == (B, N, 3)
    L = lib()
    if seq:
        name = "alif_forward_seq_staged" if seq == "staged" else "alif_forward_seq"
        rc = getattr(L, name)(B, N, T, _ptr(I), _ptr(table), _ptr(init), _ptr(spikes), _ptr(v), _ptr(a),
                              _ptr(fin), _stream(dev))
        _check(rc, name)
    else:
        rc = L.alif_forward(B, N, T, _ptr(I), _ptr(table), _ptr(init), _ptr(spikes), _ptr(v), _ptr(a),
                            _ptr(ckpt), _ptr(fin), _stream(dev))
        _check(rc, "alif_forward")
    return dict(spikes=spikes, v=v, a=a, ckpt=ckpt, final=fin)


def forward_recurrent(I_ff: torch.Tensor, W_rec_t: torch.Tensor, table: torch.Tensor, dt_ms: float, arp_ms: float,
                      init=None, want_ckpt=True, want_final=True, in_place=False, out_I=None):
    """Recurrent layer, latency D = T_R (alif_forward_recurrent).  I_ff: float32 [B, N, T];
    W_rec_t: W_rec transposed [N, N] (transpose_weights(W_rec)).  Returns dict(spikes, ckpt,
    final, I_total) with I_total = I_ff + W_rec S[t - T_R] (I_ff itself when in_place)."""
    _f32(I_ff)
    _f32(W_rec_t)
    B, N, T = I_ff.shape
    assert tuple(W_rec_t.shape) == (N, N)
    dev = I_ff.device
    spikes = torch.empty((B, N, (T + 31) // 32), dtype=torch.int32, device=dev)
    ckpt = torch.empty((B, N, max(ckpt_count(T), 1), 3), dtype=torch.int32, device=dev) if want_ckpt else None
    fin = torch.empty((B, N, 3), dtype=torch.int32, device=dev) if want_final else None
    I_total = I_ff if in_place else (out_I if out_I is not None else torch.empty_like(I_ff))
    if init is not None:
        assert init.dtype == torch.int32 and tuple(init.shape) == (B, N, 3)
    rc = lib().alif_forward_recurrent(B, N, T, _ptr(I_ff), _ptr(W_rec_t), _ptr(table), float(dt_ms), float(arp_ms),
                                      _ptr(init), _ptr(I_total), _ptr(spikes), _ptr(ckpt), _ptr(fin), _stream(dev))
    _check(rc, "alif_forward_recurrent")
    return dict(spikes=spikes, ckpt=ckpt, final=fin, I_total=I_total)


def delay_spikes(spikes: torch.Tensor, T: int, D: int) -> torch.Tensor:
    """Spike bits [B, N, ceil(T/32)] delayed by D steps (alif_delay_spikes)."""
    B, N, nw = spikes.shape
    out = torch.empty_like(spikes)
    _check(lib().alif_delay_spikes(B, N, T, int(D), _ptr(spikes), _ptr(out), _stream(spikes.device)),
           "alif_delay_spikes")
    return out


def forward_into(I, table, spikes, v=None, a=None, ckpt=None, final=None, init=None, seq=False):
    """Block (or sequential: seq=True plain, seq="staged") forward into caller-provided tensors;
    allocates nothing."""
    B, N, T = I.shape
    L = lib()
    if seq:
        name = "alif_forward_seq_staged" if seq == "staged" else "alif_forward_seq"
        rc = getattr(L, name)(B, N, T, _ptr(I), _ptr(table), _ptr(init), _ptr(spikes), _ptr(v), _ptr(a),
                              _ptr(final), _stream(I.device))
        _check(rc, name)
    else:
        rc = L.alif_forward(B, N, T, _ptr(I), _ptr(table), _ptr(init), _ptr(spikes), _ptr(v), _ptr(a),
                            _ptr(ckpt), _ptr(final), _stream(I.device))
        _check(rc, "alif_forward")


def forward_fused(S_words, W, bias, table, T, max_events_per_word=256, init=None, out_I=None, out_spikes=None,
                  out_ckpt=None, out_final=None, workspace=None):
    """alif_forward_fused: projection (exact FP32 weights, event-driven) fused into the block
    forward.  S_words [B, Nin, ceil(T/32)] input bits, W [N, Nin] FP32.  Returns dict(I, spikes,
    ckpt, final)."""
    B, Nin = S_words.shape[0], S_words.shape[1]
    N = W.shape[0]
    dev = W.device
    _f32(W, (N, Nin))
    I = out_I if out_I is not None else torch.empty((B, N, T), dtype=torch.float32, device=dev)
    spikes = out_spikes if out_spikes is not None else torch.empty((B, N, (T + 31) // 32), dtype=torch.int32, device=dev)
    ckpt = out_ckpt if out_ckpt is not None else torch.empty((B, N, ckpt_count(T), 3), dtype=torch.int32, device=dev)
    final = out_final if out_final is not None else torch.empty((B, N, 3), dtype=torch.int32, device=dev)
    L = lib()
    wsz = int(L.alif_forward_fused_workspace_size(B, Nin, T, int(max_events_per_word)))
    if workspace is None or workspace.numel() * workspace.element_size() < wsz:
        workspace = torch.empty(max(wsz, 256), dtype=torch.uint8, device=dev)
    _check(L.alif_forward_fused(B, Nin, N, int(T), _ptr(W), _ptr(S_words), _ptr(bias), _ptr(table), _ptr(init),
                                int(max_events_per_word), _ptr(I), _ptr(spikes), _ptr(ckpt), _ptr(final),
                                _ptr(workspace), wsz, _stream(dev)), "alif_forward_fused")
    return {"I": I, "spikes": spikes, "ckpt": ckpt, "final": final}


def unpack_spikes(words: torch.Tensor, T: int) -> torch.Tensor:
    """int32 [..., W] bit words -> uint8 [..., T] (bit t%32 of word t//32)."""
    w = words.to(torch.int64) & 0xFFFFFFFF
    shifts = torch.arange(32, device=words.device, dtype=torch.int64)
    bits = (w.unsqueeze(-1) >> shifts) & 1
    return bits.reshape(*words.shape[:-1], -1)[..., :T].to(torch.uint8)


# -------------------------------------------------------------- backward pass
def workspace_size(B: int, N: int) -> int:
    return int(lib().alif_backward_workspace_size(B, N))


SURROGATES = {"fast_sigmoid": 0, "multi_gaussian": 1, "boxcar": 2}


def backward(I, table, spikes, grad_spikes, ckpt=None, v_trace=None, a_trace=None, grad_v=None,
             grad_a=None, grad_final=None, init=None, slope=25.0, want_gI=True, want_ginit=False,
             seq=False, workspace=None, out_gI=None, out_gp=None, out_ginit=None, surrogate="fast_sigmoid",
             attached=False):
    """Surrogate-gradient backward.  Block version needs `ckpt` from forward(); the sequential
    version (seq=True, fast sigmoid, detached only) needs the full v_trace / a_trace.
    surrogate: "fast_sigmoid" (slope k), "multi_gaussian" or "boxcar".  attached: S[t] also
    carries its surrogate gradient through the reset of V[t+1] and the update of a[t+1]
    (alif_backward_attached); then grad_final and grad_init have 3 channels (dL/dv, dL/da,
    and the input term of dL/dS that crosses a call boundary).  Returns (grad_I, grad_init,
    grad_params [5, N])."""
    _f32(I)
    B, N, T = I.shape
    dev = I.device
    _f32(grad_spikes, (B, N, T))
    gI = out_gI if out_gI is not None else (torch.empty_like(I) if want_gI else None)
    nch = 3 if attached else 2
    ginit = out_ginit if out_ginit is not None else (
        torch.empty((B, N, nch), dtype=torch.float32, device=dev) if want_ginit else None)
    gp = out_gp if out_gp is not None else torch.empty((NUM_PARAM_GRADS, N), dtype=torch.float32, device=dev)
    wsz = workspace_size(B, N)
    if workspace is None or workspace.numel() * workspace.element_size() < wsz:
        workspace = torch.empty(max(wsz, 4), dtype=torch.uint8, device=dev)
    L = lib()
    if seq and (surrogate != "fast_sigmoid" or attached):
        raise AlifError("the sequential comparator implements the detached fast-sigmoid gradient only")
    if seq:
        rc = L.alif_backward_seq(B, N, T, _ptr(I), _ptr(table), _ptr(init), _ptr(spikes), _ptr(v_trace),
                                 _ptr(a_trace), _ptr(grad_spikes), _ptr(grad_v), _ptr(grad_a),
                                 _ptr(grad_final), float(slope), _ptr(gI), _ptr(ginit), _ptr(gp),
                                 _ptr(workspace), wsz, _stream(dev))
        _check(rc, "alif_backward_seq")
    else:
        if attached:
            # 3-channel state gradients <-> the ABI's [B, N, 2] + [B, N]
            gf2 = gfs = None
            if grad_final is not None:
                _f32(grad_final, (B, N, 3))
                gf2, gfs = grad_final[..., :2].contiguous(), grad_final[..., 2].contiguous()
            gi2 = torch.empty((B, N, 2), dtype=torch.float32, device=dev) if ginit is not None else None
            gis = torch.empty((B, N), dtype=torch.float32, device=dev) if ginit is not None else None
            rc = L.alif_backward_attached(B, N, T, _ptr(I), _ptr(table), _ptr(init), _ptr(spikes), _ptr(ckpt),
                                          _ptr(grad_spikes), _ptr(grad_v), _ptr(grad_a), _ptr(gf2), _ptr(gfs),
                                          SURROGATES[surrogate], float(slope), _ptr(gI), _ptr(gi2), _ptr(gis),
                                          _ptr(gp), _ptr(workspace), wsz, _stream(dev))
            _check(rc, "alif_backward_attached")
            if ginit is not None:
                ginit[..., :2] = gi2
                ginit[..., 2] = gis
        else:
            rc = L.alif_backward_surrogate(B, N, T, _ptr(I), _ptr(table), _ptr(init), _ptr(spikes), _ptr(ckpt),
                                           _ptr(grad_spikes), _ptr(grad_v), _ptr(grad_a), _ptr(grad_final),
                                           SURROGATES[surrogate], float(slope), _ptr(gI), _ptr(ginit), _ptr(gp),
                                           _ptr(workspace), wsz, _stream(dev))
            _check(rc, "alif_backward_surrogate")
    return gI, ginit, gp


def backward_noalloc(I, table, spikes, grad_spikes, ckpt=None, grad_v=None, grad_a=None, grad_final=None,
                     init=None, slope=25.0, out_gI=None, out_ginit=None, out_gp=None):
    """alif_backward_noalloc: the block backward with no workspace (the library's own fixed
    scratch; B*N <= 65536).  Outputs are caller-provided tensors (none allocated here when
    given).  Returns (grad_I, grad_init, grad_params)."""
    B, N, T = I.shape
    fn = getattr(lib(), "alif_backward_noalloc", None)
    if fn is None:
        raise AlifError("alif_backward_noalloc is not in the loaded library")
    if out_gp is None:
        out_gp = torch.empty((NUM_PARAM_GRADS, N), dtype=torch.float32, device=I.device)
    rc = fn(B, N, T, _ptr(I), _ptr(table), _ptr(init), _ptr(spikes), _ptr(ckpt), _ptr(grad_spikes),
            _ptr(grad_v), _ptr(grad_a), _ptr(grad_final), float(slope), _ptr(out_gI), _ptr(out_ginit),
            _ptr(out_gp), _stream(I.device))
    _check(rc, "alif_backward_noalloc")
    return out_gI, out_ginit, out_gp


# ------------------------------------------------------------------- status
def device_status(device=None) -> int:
    v = ctypes.c_int32(0)
    _check(lib().alif_device_status(_stream(device), ctypes.byref(v)), "alif_device_status")
    return v.value


def forward_stats(device=None):
    out = (ctypes.c_int64 * 4)()
    _check(lib().alif_forward_stats(_stream(device), out), "alif_forward_stats")
    return dict(exact_checks=out[0], exact_spikes=out[1], rows=out[2])


PROJ_K_ALIGN = 64


def split_bf16(W: torch.Tensor, ldw: int | None = None):
    """FP32 weights [N, Nin] -> (hi, lo) BF16 bit patterns as int16 [N, ldw] (zero padded,
    ldw defaults to Nin rounded up to 64): hi = bf16(W), lo = bf16(W - hi)."""
    _f32(W)
    N, Nin = W.shape
    if ldw is None:
        ldw = max(PROJ_K_ALIGN, -(-Nin // PROJ_K_ALIGN) * PROJ_K_ALIGN)
    hi = torch.empty((N, ldw), dtype=torch.int16, device=W.device)
    lo = torch.empty((N, ldw), dtype=torch.int16, device=W.device)
    _check(lib().syn_split_bf16(_ptr(W), N, Nin, ldw, _ptr(hi), _ptr(lo), _stream(W.device)), "syn_split_bf16")
    return hi, lo


def syn_project(S_words: torch.Tensor, W_hi: torch.Tensor, W_lo: torch.Tensor, bias=None, Nin=None, T=None,
                out=None):
    """I[b, i, t] = bias_i + sum_j W[i, j] S[b, j, t] on the tensor cores.
    S_words: int32 [B, Nin, ceil(T/32)] spike bits; W_hi/W_lo from split_bf16."""
    B, Nin_s, nw = S_words.shape
    Nin = Nin_s if Nin is None else Nin
    T = nw * 32 if T is None else T
    N, ldw = W_hi.shape
    if out is None:
        out = torch.empty((B, N, T), dtype=torch.float32, device=S_words.device)
    _check(lib().syn_project(B, Nin, N, T, _ptr(W_hi), _ptr(W_lo), ldw, _ptr(S_words), _ptr(bias), _ptr(out),
                             _stream(S_words.device)), "syn_project")
    return out


def syn_project_backward(S_words, grad_I, W=None, Nin=None, want_gW=True, want_gS=False, want_gb=True):
    """Gradients of I = W S + bias: (grad_W [N, Nin], grad_Sin [B, Nin, T], grad_bias [N])."""
    B, N, T = grad_I.shape
    Nin = S_words.shape[1] if Nin is None else Nin
    dev = grad_I.device
    gW = torch.empty((N, Nin), dtype=torch.float32, device=dev) if want_gW else None
    gS = torch.empty((B, Nin, T), dtype=torch.float32, device=dev) if want_gS else None
    gb = torch.empty((N,), dtype=torch.float32, device=dev) if want_gb else None
    wsz = int(lib().syn_project_backward_workspace_size(B, N, Nin))
    ws = torch.empty(max(wsz, 4), dtype=torch.uint8, device=dev)
    _check(lib().syn_project_backward(B, Nin, N, T, _ptr(W), _ptr(S_words), _ptr(grad_I), _ptr(gW), _ptr(gS),
                                      _ptr(gb), _ptr(ws), wsz, _stream(dev)), "syn_project_backward")
    return gW, gS, gb


def spikes_to_float(words: torch.Tensor, T: int) -> torch.Tensor:
    """Spike bits [..., ceil(T/32)] -> float32 0/1 [..., T] (library kernel)."""
    lead = words.shape[:-1]
    rows = int(np.prod(lead)) if lead else 1
    out = torch.empty((*lead, T), dtype=torch.float32, device=words.device)
    _check(lib().alif_unpack_spikes(rows, T, _ptr(words), _ptr(out), _stream(words.device)), "alif_unpack_spikes")
    return out


def vanrossum_forward(x_words, y_words, T, dt_ms, tau_ms, chunk, f_ckpt=None, loss=None):
    """Squared van Rossum distance per row (and f entering each chunk)."""
    rows = x_words.shape[0] if x_words.dim() == 2 else int(np.prod(x_words.shape[:-1]))
    _check(lib().alif_vanrossum_forward(rows, int(T), _ptr(x_words), _ptr(y_words), float(dt_ms), float(tau_ms),
                                        int(chunk), _ptr(f_ckpt), _ptr(loss), _stream(x_words.device)),
           "alif_vanrossum_forward")
    return loss


def vanrossum_backward(x_words, y_words, T, dt_ms, tau_ms, t0, t1, f_start, g_carry, grad):
    """dL/dx on steps [t0, t1) into grad [rows, t1 - t0]; g_carry updated in place."""
    rows = x_words.shape[0] if x_words.dim() == 2 else int(np.prod(x_words.shape[:-1]))
    _check(lib().alif_vanrossum_backward(rows, int(T), _ptr(x_words), _ptr(y_words), float(dt_ms), float(tau_ms),
                                         int(t0), int(t1), _ptr(f_start), _ptr(g_carry), _ptr(grad),
                                         _stream(x_words.device)), "alif_vanrossum_backward")
    return grad


def pack_spikes(S: torch.Tensor) -> torch.Tensor:
    """Float 0/1 spikes [..., T] -> int32 bit words [..., ceil(T/32)] (library kernel)."""
    _f32(S)
    T = S.shape[-1]
    lead = S.shape[:-1]
    rows = int(np.prod(lead)) if lead else 1
    out = torch.empty((*lead, (T + 31) // 32), dtype=torch.int32, device=S.device)
    _check(lib().alif_pack_spikes(rows, T, _ptr(S), _ptr(out), _stream(S.device)), "alif_pack_spikes")
    return out


def readout_weights(T: int, dt_ms: float, tau_ms: float, device) -> tuple[torch.Tensor, float]:
    """w_t = 1 - beta_o^(T-t) for t = 0..T-1 (beta_o = exp(-DT/tau), FP64 on the host, rounded
    to FP32) and their sum: the weight of step t in the leaky readout's time sum."""
    w = np.empty(max(int(T), 1), np.float32)
    s = ctypes.c_double(0.0)
    _check(lib().alif_readout_weights(int(T), float(dt_ms), float(tau_ms), w.ctypes.data_as(ctypes.c_void_p),
                                      ctypes.byref(s)), "alif_readout_weights")
    return torch.from_numpy(w[: int(T)]).to(device), float(s.value)


def readout_forward(spikes: torch.Tensor, T: int, W: torch.Tensor, bias, w_t: torch.Tensor, w_sum: float):
    """Leaky readout: spikes [B, K, ceil(T/32)] bits, W [C, K] -> (logits [B, C], counts [B, K])."""
    B, K = spikes.shape[0], spikes.shape[1]
    C = W.shape[0]
    _f32(W, (C, K))
    counts = torch.empty((B, K), dtype=torch.float32, device=W.device)
    out = torch.empty((B, C), dtype=torch.float32, device=W.device)
    _check(lib().alif_readout_forward(B, K, C, int(T), _ptr(spikes), _ptr(W), _ptr(bias), _ptr(w_t), float(w_sum),
                                      _ptr(counts), _ptr(out), _stream(W.device)), "alif_readout_forward")
    return out, counts


def readout_backward(W, w_t, w_sum, counts, grad_out, T, want_spikes=True, want_W=True, want_bias=True):
    """Backward of readout_forward -> (grad_spikes [B, K, T] float, grad_W [C, K], grad_bias [C])."""
    B, K = counts.shape
    C = W.shape[0]
    dev = W.device
    gS = torch.empty((B, K, T), dtype=torch.float32, device=dev) if want_spikes else None
    gW = torch.empty((C, K), dtype=torch.float32, device=dev) if want_W else None
    gb = torch.empty((C,), dtype=torch.float32, device=dev) if want_bias else None
    _check(lib().alif_readout_backward(B, K, C, int(T), _ptr(W), _ptr(w_t), float(w_sum), _ptr(counts),
                                       _ptr(grad_out.contiguous()), _ptr(gS), _ptr(gW), _ptr(gb), _stream(dev)),
           "alif_readout_backward")
    return gS, gW, gb


def cross_entropy(logits: torch.Tensor, labels: torch.Tensor, want_grad=True):
    """Mean softmax cross-entropy -> (loss [1], grad_logits [B, C] or None)."""
    _f32(logits)
    B, C = logits.shape
    assert labels.dtype == torch.int32 and labels.shape == (B,)
    dev = logits.device
    loss = torch.empty((1,), dtype=torch.float32, device=dev)
    g = torch.empty_like(logits) if want_grad else None
    ws = torch.empty((B,), dtype=torch.float32, device=dev)
    _check(lib().alif_cross_entropy(B, C, _ptr(logits), _ptr(labels), _ptr(loss), _ptr(g), _ptr(ws), _stream(dev)),
           "alif_cross_entropy")
    return loss, g


def transpose_weights(W: torch.Tensor) -> torch.Tensor:
    """FP32 weights [N, Nin] -> W_t [Nin, N] (library kernel), the layout of syn_project_events."""
    _f32(W)
    N, Nin = W.shape
    Wt = torch.empty((Nin, N), dtype=torch.float32, device=W.device)
    _check(lib().syn_transpose_weights(_ptr(W), N, Nin, _ptr(Wt), _stream(W.device)), "syn_transpose_weights")
    return Wt


def syn_project_events(S_words: torch.Tensor, W_t: torch.Tensor, bias=None, Nin=None, T=None, out=None):
    """Event-driven I[b, i, t] = bias_i + sum_{active j} W[i, j] from spike bits [B, Nin, ceil(T/32)]
    and W_t [Nin, N] (exact FP32 weights)."""
    B, Nin_s, nw = S_words.shape
    Nin = Nin_s if Nin is None else Nin
    T = nw * 32 if T is None else T
    N = W_t.shape[1]
    if out is None:
        out = torch.empty((B, N, T), dtype=torch.float32, device=S_words.device)
    _check(lib().syn_project_events(B, Nin, N, T, _ptr(W_t), _ptr(S_words), _ptr(bias), _ptr(out),
                                    _stream(S_words.device)), "syn_project_events")
    return out
