"""ctypes front end of the FP64 ALIF oracle (oracle/alif_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
bench's CPU-baseline leg.  The product path never imports this module.

The C file is the standard step-by-step ALIF model (Eqs 1-5, Section 2) in
double precision with its surrogate-gradient BPTT (Supplementary, "Surrogate
gradient", "Detaching gradients"), and the recurrent layer with transmission
latency D = T_R (Eq 3's recurrent term).  `build()` compiles it with gcc.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "alif_oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lib = None

NEVER = np.iinfo(np.int64).max


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_liboracle.so (plain gcc, -O2, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
                               "-ffp-contract=off", "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i64, dbl, cint = ctypes.c_int64, ctypes.c_double, ctypes.c_int
        lib.oracle_tr.argtypes = [dbl, dbl]
        lib.oracle_tr.restype = i64
        lib.oracle_alif_forward.argtypes = [i64, i64, i64, P, P, P, P, P, P, dbl, dbl,
                                            P, P, P, P, P, P, P, P, P, P, P, P, P, P, cint]
        lib.oracle_alif_forward.restype = cint
        lib.oracle_alif_backward.argtypes = [i64, i64, i64, P, P, P, P, P, P, dbl, dbl, dbl, cint, cint,
                                             P, P, P, P, P, P, P, P, P, P, P, P, P, P, P, P, cint]
        lib.oracle_alif_backward.restype = cint
        lib.oracle_alif_forward_recurrent.argtypes = [i64, i64, i64, P, P, P, P, P, P, P, dbl, dbl,
                                                      P, P, P, P, P, P, cint]
        lib.oracle_alif_forward_recurrent.restype = cint
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def tr(dt: float, arp: float) -> int:
    """T_R = ARP/DT as an integer (Section 3.2), or -1 when not an integer >= 1."""
    return int(_load().oracle_tr(float(dt), float(arp)))


@dataclass
class Params:
    """Per-neuron parameters [N] (promoted exactly to float64)."""
    tau_mem: np.ndarray
    tau_adapt: np.ndarray
    theta0: np.ndarray
    d: np.ndarray
    R: np.ndarray | None = None

    def arrays(self):
        f = lambda x: None if x is None else np.ascontiguousarray(x, dtype=np.float64)
        return f(self.tau_mem), f(self.tau_adapt), f(self.theta0), f(self.d), f(self.R)


@dataclass
class Init:
    """Initial condition at t = 0 in the paper's variables, per row [B*N]."""
    V: np.ndarray | None = None
    S: np.ndarray | None = None
    a: np.ndarray | None = None
    C: np.ndarray | None = None


@dataclass
class Forward:
    S: np.ndarray       # uint8 [B,N,T]
    V: np.ndarray       # float64 [B,N,T]
    a: np.ndarray       # float64 [B,N,T]
    theta: np.ndarray   # float64 [B,N,T]
    mask: np.ndarray    # uint8 [B,N,T]  (Eq 4 admission)
    final_V: np.ndarray
    final_S: np.ndarray
    final_a: np.ndarray
    final_C: np.ndarray

    @property
    def margin(self):
        return self.V - self.theta


def _init_arrays(init: Init | None, rows: int):
    if init is None:
        return None, None, None, None
    V = None if init.V is None else np.ascontiguousarray(init.V, dtype=np.float64).reshape(rows)
    S = None if init.S is None else np.ascontiguousarray(init.S, dtype=np.uint8).reshape(rows)
    a = None if init.a is None else np.ascontiguousarray(init.a, dtype=np.float64).reshape(rows)
    C = None if init.C is None else np.ascontiguousarray(init.C, dtype=np.int64).reshape(rows)
    return V, S, a, C


def forward(I: np.ndarray, params: Params, dt: float, arp: float, init: Init | None = None,
            force: np.ndarray | None = None, nthreads: int = 1, records: bool = True) -> Forward:
    """Run Eqs 1-5 step by step.  I: float32 [B,N,T].  force: int8 [B,N,T] with -1 = free,
    0/1 = impose that spike decision (teacher forcing after a permitted near-tie flip)."""
    lib = _load()
    I = np.ascontiguousarray(I, dtype=np.float32)
    B, N, T = I.shape
    rows = B * N
    tm, ta, th0, d, R = params.arrays()
    iV, iS, ia, iC = _init_arrays(init, rows)
    if force is not None:
        force = np.ascontiguousarray(force, dtype=np.int8)
        assert force.shape == I.shape
    S = np.zeros((B, N, T), np.uint8)
    if records:
        V = np.zeros((B, N, T)); a = np.zeros((B, N, T)); th = np.zeros((B, N, T))
        m = np.zeros((B, N, T), np.uint8)
    else:
        V = a = th = m = None
    fV = np.zeros(rows); fS = np.zeros(rows, np.uint8); fa = np.zeros(rows)
    fC = np.zeros(rows, np.int64)
    rc = lib.oracle_alif_forward(B, N, T, _p(I), _p(tm), _p(ta), _p(th0), _p(d), _p(R),
                                 float(dt), float(arp), _p(iV), _p(iS), _p(ia), _p(iC),
                                 _p(force), _p(S), _p(V), _p(a), _p(th), _p(m),
                                 _p(fV), _p(fS), _p(fa), _p(fC), int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle_alif_forward rejected its arguments (code {rc})")
    return Forward(S, V, a, th, m, fV.reshape(B, N), fS.reshape(B, N), fa.reshape(B, N),
                   fC.reshape(B, N))


@dataclass
class Backward:
    gI: np.ndarray | None       # [B,N,T]
    g_tau_mem: np.ndarray       # per row [B,N]
    g_tau_adapt: np.ndarray
    g_theta0: np.ndarray
    g_d: np.ndarray
    g_R: np.ndarray
    g_V0: np.ndarray
    g_a0: np.ndarray


SURROGATES = {"fast_sigmoid": 0, "multi_gaussian": 1, "boxcar": 2}


def backward(I: np.ndarray, params: Params, dt: float, arp: float, gS: np.ndarray,
             gV: np.ndarray | None = None, ga: np.ndarray | None = None, slope: float = 25.0,
             init: Init | None = None, force: np.ndarray | None = None,
             want_gI: bool = True, nthreads: int = 1, surrogate: str = "fast_sigmoid",
             attached: bool = False) -> Backward:
    """Surrogate-gradient BPTT of `forward`; surrogate "fast_sigmoid" (slope k),
    "multi_gaussian" or "boxcar" (Supplementary, "Surrogate gradient").  Detached by
    default; `attached` also carries dL/dS[t] through the reset factor of V[t+1] and the
    update of a[t+1] (Supplementary, "Detaching gradients")."""
    lib = _load()
    I = np.ascontiguousarray(I, dtype=np.float32)
    B, N, T = I.shape
    rows = B * N
    tm, ta, th0, d, R = params.arrays()
    iV, iS, ia, iC = _init_arrays(init, rows)
    f64 = lambda x: None if x is None else np.ascontiguousarray(x, dtype=np.float64).reshape(B, N, T)
    gS, gV, ga = f64(gS), f64(gV), f64(ga)
    if force is not None:
        force = np.ascontiguousarray(force, dtype=np.int8)
    gI = np.zeros((B, N, T)) if want_gI else None
    outs = [np.zeros(rows) for _ in range(7)]
    rc = lib.oracle_alif_backward(B, N, T, _p(I), _p(tm), _p(ta), _p(th0), _p(d), _p(R),
                                  float(dt), float(arp), float(slope), SURROGATES[surrogate], int(bool(attached)),
                                  _p(iV), _p(iS), _p(ia), _p(iC), _p(force),
                                  _p(gS), _p(gV), _p(ga), _p(gI), *[_p(o) for o in outs],
                                  int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle_alif_backward rejected its arguments (code {rc})")
    outs = [o.reshape(B, N) for o in outs]
    return Backward(gI, *outs)


@dataclass
class RecurrentForward:
    S: np.ndarray        # uint8 [B,N,T]
    V: np.ndarray        # float64 [B,N,T]
    a: np.ndarray        # float64 [B,N,T]
    theta: np.ndarray    # float64 [B,N,T]
    mask: np.ndarray     # uint8 [B,N,T]
    I_total: np.ndarray  # float64 [B,N,T]: I_ff + sum_j W_rec[i,j] S_j[t - T_R]

    @property
    def margin(self):
        return self.V - self.theta


def forward_recurrent(I_ff: np.ndarray, W_rec: np.ndarray, params: Params, dt: float, arp: float,
                      nthreads: int = 1) -> RecurrentForward:
    """Recurrent layer with transmission delay D = T_R (Section 2, Eq 3's recurrent term):
    every neuron of a batch element stepped together through Eqs 1-5 with
    I[t] = I_ff[t] + W_rec S[t - T_R].  I_ff: float32 [B,N,T]; W_rec: float32 [N,N]."""
    lib = _load()
    I_ff = np.ascontiguousarray(I_ff, dtype=np.float32)
    W_rec = np.ascontiguousarray(W_rec, dtype=np.float32)
    B, N, T = I_ff.shape
    assert W_rec.shape == (N, N)
    tm, ta, th0, d, R = params.arrays()
    S = np.zeros((B, N, T), np.uint8)
    V = np.zeros((B, N, T)); a = np.zeros((B, N, T)); th = np.zeros((B, N, T))
    m = np.zeros((B, N, T), np.uint8); It = np.zeros((B, N, T))
    rc = lib.oracle_alif_forward_recurrent(B, N, T, _p(I_ff), _p(W_rec), _p(tm), _p(ta), _p(th0), _p(d),
                                           _p(R), float(dt), float(arp), _p(S), _p(V), _p(a), _p(th),
                                           _p(m), _p(It), int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle_alif_forward_recurrent rejected its arguments (code {rc})")
    return RecurrentForward(S, V, a, th, m, It)
