"""Seeded synthetic inputs for the Fisher-vector encoder.

This module only draws random numbers: GMM parameters and descriptor sets
shaped like the dense-grid workloads of the paper (Sec. 4: K=256 diagonal
components, dense descriptors at stride 4 over an 8-scale pyramid of a
320x240 frame, which gives 80x60x4 = 19200 descriptors). It holds none of
the encoder's arithmetic, so both the GPU path and the CPU oracle can take
their inputs from it without sharing any of the method.

Recipe (all draws from numpy's PCG64 seeded by a SeedSequence built from
(base_seed, stream, index), so every frame of every workload is reproducible
on its own):

* weights   w ~ Dirichlet(1)   (normalised Exp(1) draws)
* means     mu ~ N(0, 1)
* variances sigma^2 ~ Uniform(0.1, 1.0)
* descriptors: a fraction `gmm_frac` drawn from the GMM itself
  (component k ~ w, then x ~ N(mu_k, diag sigma^2_k)), the rest Uniform(-3, 3)
  outliers, rows shuffled.
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 20160603

# Stream identifiers keep the GMM and descriptor draws of different workloads
# independent of one another.
STREAM_GMM = 1
STREAM_FRAMES = 2
STREAM_SIZES = 3
STREAM_ARRIVALS = 4
STREAM_SIFT = 5
STREAM_PCA = 6
STREAM_IMAGES = 7


def _rng(*key: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([BASE_SEED, *key])))


def make_gmm(K: int, D: int, seed: int = 0, var_lo: float = 0.1, var_hi: float = 1.0):
    """Return (w[K], mu[K,D], var[K,D]) as float32 arrays.

    The weights are renormalised in float64 and then rounded to float32, so
    their float32 sum is 1 within a few ulps.
    """
    g = _rng(STREAM_GMM, seed, K, D)
    e = g.standard_exponential(K)
    w = (e / e.sum()).astype(np.float32)
    mu = g.standard_normal((K, D)).astype(np.float32)
    var = g.uniform(var_lo, var_hi, size=(K, D)).astype(np.float32)
    return w, mu, var


def sample_descriptors(w, mu, var, N: int, seed: int = 0, gmm_frac: float = 1.0,
                       lo: float = -3.0, hi: float = 3.0) -> np.ndarray:
    """Draw N descriptors (float32, N x D): gmm_frac of them from the GMM, the
    rest Uniform(lo, hi) outliers, in shuffled order."""
    K, D = mu.shape
    g = _rng(STREAM_FRAMES, seed, N, K, D)
    n_gmm = int(round(N * gmm_frac))
    p = np.asarray(w, dtype=np.float64)
    p = p / p.sum()
    comp = g.choice(K, size=n_gmm, p=p)
    z = g.standard_normal((n_gmm, D), dtype=np.float32)
    x_gmm = mu[comp] + np.sqrt(var[comp]) * z
    x_out = g.uniform(lo, hi, size=(N - n_gmm, D)).astype(np.float32)
    X = np.concatenate([x_gmm.astype(np.float32), x_out], axis=0)
    g.shuffle(X, axis=0)
    return np.ascontiguousarray(X, dtype=np.float32)


def frame_sizes(B: int, lo: int, hi: int, seed: int = 0) -> np.ndarray:
    """B per-frame descriptor counts drawn Uniform{lo..hi} (inclusive)."""
    g = _rng(STREAM_SIZES, seed, B, lo, hi)
    return g.integers(lo, hi + 1, size=B).astype(np.int64)


def arrival_times(n_streams: int, fps: float, seconds: float, jitter_mean_s: float = 0.005,
                  seed: int = 0) -> np.ndarray:
    """Frame arrival times (seconds) for n_streams periodic video streams with
    exponential (Poisson-process) jitter clipped to one frame period.

    Returns an array of shape (n_frames_total, 3): (time, stream_id, frame_idx),
    sorted by time."""
    g = _rng(STREAM_ARRIVALS, seed, n_streams)
    period = 1.0 / fps
    n = int(round(seconds * fps))
    rows = []
    for s in range(n_streams):
        phase = g.uniform(0.0, period)
        jit = np.minimum(g.exponential(jitter_mean_s, size=n), period)
        t = phase + np.arange(n) * period + jit
        rows.append(np.stack([t, np.full(n, s), np.arange(n)], axis=1))
    a = np.concatenate(rows, axis=0)
    return a[np.argsort(a[:, 0], kind="stable")]


def to_bf16_grid(X: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even) and return
    them as float32. Used to hand both the GPU and the oracle the identical
    input when the encoder stores descriptors as bfloat16."""
    a = np.ascontiguousarray(X, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (a >> 16) & 1
    r = ((a + 0x7FFF + lsb) >> 16) << 16
    return (r.astype(np.uint32)).view(np.float32).reshape(X.shape)


def sample_sift_like(N: int, Din: int = 128, seed: int = 0) -> np.ndarray:
    """N raw descriptors shaped like SIFT histograms (float32, N x Din):
    non-negative gradient-orientation mass with a few dominant bins per
    descriptor, unit L2 norm, entries capped at 0.2 and renormalised (the
    normalisation SIFT descriptors carry)."""
    g = _rng(STREAM_SIFT, seed, N, Din)
    base = g.gamma(0.6, 1.0, size=(N, Din))
    x = base / np.maximum(np.linalg.norm(base, axis=1, keepdims=True), 1e-12)
    x = np.minimum(x, 0.2)
    x = x / np.maximum(np.linalg.norm(x, axis=1, keepdims=True), 1e-12)
    return np.ascontiguousarray(x, dtype=np.float32)


def make_pca(Din: int = 128, m: int = 62, seed: int = 0):
    """A synthetic PCA: (basis m x Din with orthonormal rows drawn uniformly,
    mean Din) as float32. The basis comes from the QR factor of a Gaussian
    matrix (a random rotation), the mean ~ U(0, 0.15) like SIFT entries."""
    g = _rng(STREAM_PCA, seed, Din, m)
    q, r = np.linalg.qr(g.standard_normal((Din, m)))
    q = q * np.sign(np.diag(r))[None, :]
    mean = g.uniform(0.0, 0.15, size=Din)
    return np.ascontiguousarray(q.T, dtype=np.float32), mean.astype(np.float32)


def sample_positions(N: int, seed: int = 0) -> np.ndarray:
    """Normalised (x, y) positions of N descriptors, Uniform(-0.5, 0.5)^2."""
    g = _rng(STREAM_IMAGES, seed, N)
    return np.ascontiguousarray(g.uniform(-0.5, 0.5, size=(N, 2)), dtype=np.float32)


def make_frames(B: int, H: int = 240, W: int = 320, seed: int = 0) -> np.ndarray:
    """B grey-level frames (float32, B x H x W, values in [0, 1]) with the
    structure dense SIFT responds to: 24 Gaussian blobs of random position,
    width (4-40 px) and sign, 3 oriented gratings of random period (8-48 px)
    and angle, and pixel noise of standard deviation 0.02, rescaled to [0, 1]."""
    g = _rng(STREAM_IMAGES, seed, B, H, W)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    out = np.empty((B, H, W), np.float32)
    for b in range(B):
        img = np.zeros((H, W))
        for _ in range(24):
            cy, cx = g.uniform(0, H), g.uniform(0, W)
            sd = g.uniform(4, 40)
            img += g.choice([-1.0, 1.0]) * g.uniform(0.3, 1.0) * np.exp(-((yy - cy) ** 2 + (xx - cx) ** 2) / (2 * sd * sd))
        for _ in range(3):
            th, per = g.uniform(0, np.pi), g.uniform(8, 48)
            img += 0.3 * np.sin(2 * np.pi * (np.cos(th) * xx + np.sin(th) * yy) / per + g.uniform(0, 2 * np.pi))
        img += g.normal(0, 0.02, size=(H, W))
        img = (img - img.min()) / max(img.max() - img.min(), 1e-12)
        out[b] = img
    return out
