"""Double-precision CPU oracle for Fisher-vector encoding.

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the benchmark's
CPU-baseline leg may import this package; the product path never does.

The arithmetic lives in ``fv_oracle.c`` (paper Sec. 3.1: the GMM
log-likelihoods, the posteriors and the U, V statistics of Algorithm 1, stated
from their definitions; plus the improved-FV normalisation of Sec. 4). This
module compiles it with the host C compiler, loads it with ctypes and converts
arrays. Every parity pin of the oracle is in the oracle tests; no function
here is "parity unpinned".
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


def _bind(lib):
    P = ctypes.c_void_p
    lib.fvo_encode.restype = ctypes.c_int
    lib.fvo_encode.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                               P, P, P, P, ctypes.c_double, P, P, P, P, P, P]
    lib.fvo_log_constants.restype = ctypes.c_int
    lib.fvo_log_constants.argtypes = [ctypes.c_int, ctypes.c_int, P, P, P]
    lib.fvo_log_likelihoods.restype = ctypes.c_int
    lib.fvo_log_likelihoods.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_int, P, P, P, P, P]
    lib.fvo_posteriors.restype = ctypes.c_int
    lib.fvo_posteriors.argtypes = [ctypes.c_int64, ctypes.c_int, P, P, P]
    lib.fvo_pca_project.restype = ctypes.c_int
    lib.fvo_pca_project.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_int, P, P, P, P, P]
    lib.fvo_em_step.restype = ctypes.c_int
    lib.fvo_em_step.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_int, P, P, P, P, ctypes.c_double, P, P, P, P]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(ctypes.CDLL(_SO))
    return _lib


def load_variant(src: str, out_dir: str):
    """Compile another copy of the oracle source (the tests plant mistakes
    in copies to check that the pins catch them) and return its bound
    library, for the ``lib`` argument of encode()."""
    so = os.path.join(out_dir, os.path.basename(src) + ".so")
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
                           "-ffp-contract=off", src, "-o", so, "-lm"])
    return _bind(ctypes.CDLL(so))


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def encode(X, w, mu, var, tau: float = 0.0, want_gamma: bool = False, want_stats: bool = False, lib=None):
    """Encode one descriptor set. Inputs are converted to float64 (exactly).

    Returns a dict with ``fv`` (2KD, normalised), ``fv_raw`` (2KD, before the
    signed square root and L2 step), ``status``, and optionally ``gamma``
    (N x K), ``U``, ``V`` (K x D, unscaled sums) and ``S0`` (K).
    """
    lib = lib or _load()
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


def log_likelihoods(X, w, mu, var):
    """The N x K matrix L_ik = log w_k + log N(x_i; mu_k, sigma^2_k) + (D/2) log 2pi."""
    lib = _load()
    X = np.ascontiguousarray(X, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64).reshape(-1)
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    var = np.ascontiguousarray(var, dtype=np.float64)
    K, D = mu.shape
    N = X.shape[0]
    L = np.zeros((max(N, 1), K))
    st = lib.fvo_log_likelihoods(N, D, K, _p(X), _p(w), _p(mu), _p(var), _p(L))
    assert st == 0, st
    return L[:N]


def posteriors(X, w, mu, var):
    """(gamma N x K, lse N): the posteriors and the per-descriptor
    log-sum-exp lse_i = log sum_k exp(L_ik), i.e. log p(x_i) + (D/2) log 2pi."""
    lib = _load()
    L = log_likelihoods(X, w, mu, var)
    N, K = L.shape
    g = np.zeros((max(N, 1), K))
    lse = np.zeros(max(N, 1))
    st = lib.fvo_posteriors(N, K, _p(np.ascontiguousarray(L if N else np.zeros((1, K)))), _p(g), _p(lse))
    assert st == 0, st
    return g[:N], lse[:N]


def em_step(X, w, mu, var, reg: float = 0.0):
    """One EM step of the diagonal GMM from its definitions (FP64): returns
    (w', mu', var', mean log-likelihood of X under the input model)."""
    lib = _load()
    X = np.ascontiguousarray(X, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64).reshape(-1)
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    var = np.ascontiguousarray(var, dtype=np.float64)
    K, D = mu.shape
    N = X.shape[0]
    w2, mu2, var2 = np.zeros(K), np.zeros((K, D)), np.zeros((K, D))
    ll = ctypes.c_double()
    st = lib.fvo_em_step(N, D, K, _p(X), _p(w), _p(mu), _p(var), float(reg), _p(w2), _p(mu2), _p(var2),
                         ctypes.byref(ll))
    assert st == 0, st
    return w2, mu2, var2, ll.value


def pca_project(X, basis, mean=None, xy=None):
    """Sec. 3.1's descriptor step: y_i = [basis (x_i - mean); xy_i] in FP64
    (basis m x Din, rows the principal directions; xy N x 2 or None)."""
    lib = _load()
    X = np.ascontiguousarray(X, dtype=np.float64)
    P = np.ascontiguousarray(basis, dtype=np.float64)
    m, Din = P.shape
    N = X.shape[0]
    mean = None if mean is None else np.ascontiguousarray(mean, dtype=np.float64)
    xy = None if xy is None else np.ascontiguousarray(xy, dtype=np.float64)
    D = m + (2 if xy is not None else 0)
    Y = np.zeros((max(N, 1), D))
    st = lib.fvo_pca_project(N, Din, m, _p(X if N else np.zeros((1, Din))), _p(mean), _p(P), _p(xy), _p(Y))
    assert st == 0, st
    return Y[:N]
