"""Pins of the oracle's PCA step (Sec. 3.1: PCA to m dimensions plus the
normalised X and Y position, D = m + 2), each against a fact outside it:

* with the eigenvectors of a sample covariance (numpy's eigh) as the basis,
  the projected training set has zero mean and a diagonal covariance whose
  diagonal is the eigenvalues (what PCA means);
* with an orthonormal basis spanning the data's centred subspace, the basis
  transposed maps the projection back to the centred descriptors;
* the (x, y) columns are appended unchanged after the m projected ones."""
import numpy as np

import oracle
from paper_1604_03498_gb300 import synth


def test_projection_on_principal_axes_diagonalises_the_covariance():
    X = synth.sample_sift_like(3000, 128, seed=1).astype(np.float64)
    mean = X.mean(0)
    C = np.cov(X - mean, rowvar=False, bias=True)
    ev, V = np.linalg.eigh(C)
    order = np.argsort(ev)[::-1][:20]
    P = V[:, order].T
    Y = oracle.pca_project(X, P, mean)
    np.testing.assert_allclose(Y.mean(0), 0.0, atol=1e-12)
    Cy = (Y.T @ Y) / len(Y)
    np.testing.assert_allclose(np.diag(Cy), ev[order], rtol=1e-9)
    off = Cy - np.diag(np.diag(Cy))
    assert np.abs(off).max() <= 1e-12


def test_orthonormal_round_trip_and_appended_positions():
    g = np.random.default_rng(2)
    Din, m, N = 128, 30, 200
    Q, _ = np.linalg.qr(g.standard_normal((Din, m)))
    mean = g.uniform(0, 0.1, Din)
    coef = g.standard_normal((N, m))
    X = mean + coef @ Q.T          # descriptors inside the basis' span
    xy = g.uniform(-0.5, 0.5, (N, 2))
    Y = oracle.pca_project(X, Q.T, mean, xy)
    assert Y.shape == (N, m + 2)
    np.testing.assert_allclose(Y[:, :m], coef, atol=1e-12)
    np.testing.assert_allclose(Y[:, :m] @ Q.T + mean, X, atol=1e-12)
    assert np.array_equal(Y[:, m:], xy)


def test_synthetic_pca_basis_is_orthonormal():
    P, mean = synth.make_pca(128, 62, seed=3)
    np.testing.assert_allclose(P.astype(np.float64) @ P.T.astype(np.float64), np.eye(62), atol=1e-6)
    assert mean.shape == (128,)
