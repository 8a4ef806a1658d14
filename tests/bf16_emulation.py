"""CPU model of the BF16 precision form's arithmetic (test infrastructure).

It reproduces, in float64 numpy, the roundings the fused tcgen05 encoder makes
so that the error of each one can be measured against the FP64 oracle without
a GPU:

* descriptors are bfloat16 (the caller hands the same rounded values to the
  oracle), x^2 is split exactly into bf16 hi + lo;
* the log-likelihood operands Q = mu/sigma^2 and R = -1/(2 sigma^2) are
  rounded to FP32 and split into bf16 hi + lo; the log-likelihood is the sum
  of the five split products plus the FP32-rounded constant
  c = log w - 1/2 sum log sigma^2 - 1/2 sum mu^2/sigma^2 (Sec. 3.1 expanded);
* the posteriors are rounded to bfloat16 before the statistics GEMM
  gamma^T [X | X^2hi | X^2lo | 1];
* the raw moments are centred (the encoder does it as it writes each share's
  slot; centring is linear, so one frame-wide centring stands for it here)
  and the Sec. 4 encoding is applied.

Any term can be switched off (``drop``) or the posterior rounding changed
(``gamma``: "bf16", "fp16", "hilo" for a bf16 hi + lo pair, "exact"), which
is how the error budget of each split product is measured. FP32
accumulation order inside the tensor cores is not modelled (float64 sums).
Nothing here is shared with the CUDA sources or the oracle.
"""
import numpy as np


def bf16(a):
    """Round float64/float32 values to bfloat16 (via float32, ties to even)."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def fp16(a):
    return np.asarray(a, dtype=np.float16).astype(np.float64)


def split(a):
    """FP32-rounded value as bf16 hi + bf16 lo."""
    f = np.asarray(a, dtype=np.float32).astype(np.float64)
    hi = bf16(f)
    return hi, bf16(f - hi)


def encode(X, w, mu, var, drop=(), gamma="bf16"):
    """Normalised Fisher vector (2KD, float64) of the BF16 form's arithmetic.
    X must already be on the bfloat16 grid."""
    X = np.asarray(X, np.float64)
    w = np.asarray(w, np.float64)
    mu = np.asarray(mu, np.float64)
    var = np.asarray(var, np.float64)
    N, D = X.shape
    K = mu.shape[0]
    w = w / w.sum()
    p = 1.0 / var
    q, r = mu * p, -0.5 * p
    qh, ql = split(q)
    rh, rl = split(r)
    c = np.log(w) - 0.5 * np.log(var).sum(1) - 0.5 * (mu * mu * p).sum(1)
    c = np.asarray(c * np.log2(np.e), np.float32).astype(np.float64) / np.log2(np.e)
    x2 = X * X
    x2h = bf16(x2)
    x2l = bf16(x2 - x2h)
    L = X @ qh.T
    if "xQlo" not in drop:
        L += X @ ql.T
    L += x2h @ rh.T
    if "x2hiRlo" not in drop:
        L += x2h @ rl.T
    if "x2loRhi" not in drop:
        L += x2l @ rh.T
    L += c[None, :]
    L = np.asarray(L, np.float32).astype(np.float64)     # FP32 accumulator in TMEM
    m = L.max(1, keepdims=True)
    e = np.exp(L - m)
    g = e / e.sum(1, keepdims=True)
    if gamma == "bf16":
        g = bf16(g)
    elif gamma == "fp16":
        g = fp16(g)
    elif gamma == "hilo":
        gh = bf16(g)
        g = gh + bf16(g - gh)
    S0 = g.sum(0)
    S1 = g.T @ X
    S2 = g.T @ x2h
    if "X2lo" not in drop:
        S2 = S2 + g.T @ x2l
    a = S1 - mu * S0[:, None]
    b = S2 - mu * S1
    M2 = b - mu * a
    u = a / np.sqrt(var) / (N * np.sqrt(w))[:, None]
    v = (M2 / var - S0[:, None]) / (N * np.sqrt(2 * w))[:, None]
    z = np.concatenate([u.ravel(), v.ravel()])
    z = np.sign(z) * np.sqrt(np.abs(z))
    n = np.linalg.norm(z)
    return z / n if n > 0 else z
