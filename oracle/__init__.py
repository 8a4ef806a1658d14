"""Double-precision CPU oracle for Fisher-vector encoding.

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the benchmark's
CPU-baseline leg may import this package; the product path never does.

The arithmetic lives in ``fv_oracle.c`` (paper Sec. 3.1, Algorithm 1, plus
the improved-FV normalisation of Sec. 4). This module compiles it with the
host C compiler, loads it with ctypes and converts arrays. Every parity pin
of the oracle is in the oracle tests; no function here is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fv_oracle.c")
_OUTDIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUTDIR, "libfv_oracle.so")
_lib = None
_lock = threading.Lock()

FVO_OK, FVO_EMPTY, FVO_BADARG, FVO_NOMEM = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle shared library (plain C, IEEE double, no fast-math)."""
    os.makedirs(_OUTDIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                               "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            P = ctypes.c_void_p
            lib.fvo_encode.restype = ctypes.c_int
            lib.fvo_encode.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                       P, P, P, P, ctypes.c_double, P, P, P, P, P, P]
            lib.fvo_log_constants.restype = ctypes.c_int
            lib.fvo_log_constants.argtypes = [ctypes.c_int, ctypes.c_int, P, P, P]
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def encode(X, w, mu, var, tau: float = 0.0, want_gamma: bool = False, want_stats: bool = False):
    """Encode one descriptor set. Inputs are converted to float64 (exactly).

    Returns a dict with ``fv`` (2KD, normalised), ``fv_raw`` (2KD, before the
    signed square root and L2 step), ``status``, and optionally ``gamma``
    (N x K), ``U``, ``V`` (K x D, unscaled sums) and ``S0`` (K).
    """
    lib = _load()
    X = np.ascontiguousarray(X, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64).reshape(-1)
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    var = np.ascontiguousarray(var, dtype=np.float64)
    K, D = mu.shape
    N = X.shape[0] if X.size else 0
    if X.size:
        assert X.shape[1] == D
    else:
        X = np.zeros((1, D), dtype=np.float64)
    fv = np.zeros(2 * K * D)
    fv_raw = np.zeros(2 * K * D)
    gamma = np.zeros((max(N, 1), K)) if want_gamma else None
    U = np.zeros((K, D)) if want_stats else None
    V = np.zeros((K, D)) if want_stats else None
    S0 = np.zeros(K) if want_stats else None
    st = lib.fvo_encode(N, D, K, _p(X), _p(w), _p(mu), _p(var), float(tau),
                        _p(fv), _p(fv_raw), _p(gamma), _p(U), _p(V), _p(S0))
    out = {"status": st, "fv": fv, "fv_raw": fv_raw}
    if want_gamma:
        out["gamma"] = gamma[:N]
    if want_stats:
        out.update(U=U, V=V, S0=S0)
    return out


def log_constants(w, var):
    """Step 1's constant of every component, log w_k - 1/2 sum_d log var_kd
    (Algorithm 1), in FP64; returns an array of K values."""
    lib = _load()
    w = np.ascontiguousarray(w, dtype=np.float64).reshape(-1)
    var = np.ascontiguousarray(var, dtype=np.float64)
    K, D = var.shape
    cst = np.zeros(K)
    st = lib.fvo_log_constants(D, K, _p(w), _p(var), _p(cst))
    assert st == 0, st
    return cst
