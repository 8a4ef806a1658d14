"""Pins of the dense SIFT oracle (Sec. 3.1-3.2), each against something
outside it:

* the separable triangular filter against scipy's 2-D correlation with the
  outer-product kernel (zero padding);
* every descriptor of small images against a brute-force sum over all
  pixels of magnitude x triangular spatial weights x the circular triangle
  weight in orientation, written from the definition (no filters, no
  separability, no channel planes);
* a linear ramp: all gradient mass in orientation 0, interior descriptors
  with 16 equal entries, 1/4 each after normalisation;
* the pyramid's scale list and sizes, bilinear resizing of a ramp, and the
  descriptor count of a 320x240 frame."""
import math

import numpy as np
import pytest

from oracle import dsift_oracle as O
from paper_1604_03498_gb300 import synth


def test_triangular_filter_matches_scipy_correlation():
    nd = pytest.importorskip("scipy.ndimage")
    g = np.random.default_rng(1)
    ch = g.random((8, 23, 31))
    for b in (2, 4, 6):
        k = O.triangle(b)
        ref = np.stack([nd.correlate(c, np.outer(k, k), mode="constant", cval=0.0) for c in ch])
        np.testing.assert_allclose(O.triangular_filter(ch, b), ref, rtol=1e-12, atol=1e-12)


def _brute_force(img, b, stride):
    gx, gy = O.gradients(img)   # pinned below through the ramp
    H, W = img.shape
    m = np.hypot(gx, gy)
    th = np.mod(np.arctan2(gy, gx), 2 * math.pi)
    t = th / (2 * math.pi / 8)
    out = []
    for y0 in range(2 * b, H - 2 * b + 1, stride):
        for x0 in range(2 * b, W - 2 * b + 1, stride):
            d = np.zeros(128)
            for by in range(4):
                for bx in range(4):
                    cy, cx = y0 + (by - 1.5) * b, x0 + (bx - 1.5) * b
                    for o in range(8):
                        dist = np.abs(t - o)
                        dist = np.minimum(dist, 8 - dist)           # circular distance in bins
                        wo = np.maximum(0.0, 1.0 - dist)
                        wy = np.maximum(0.0, 1.0 - np.abs(np.arange(H) - cy) / b)[:, None]
                        wx = np.maximum(0.0, 1.0 - np.abs(np.arange(W) - cx) / b)[None, :]
                        d[(by * 4 + bx) * 8 + o] = np.sum(wy * wx * wo * m)
            n = np.linalg.norm(d)
            if n > 0:
                d = np.minimum(d / n, 0.2)
                d = d / np.linalg.norm(d)
            out.append(d)
    return np.array(out)


@pytest.mark.parametrize("H,W,b,stride,seed", [(24, 28, 4, 4, 1), (30, 26, 4, 2, 2), (40, 40, 8, 4, 3)])
def test_descriptors_against_brute_force(H, W, b, stride, seed):
    img = synth.make_frames(1, H, W, seed=seed)[0].astype(np.float64)
    D, P = O.descriptors_of_image(img, b, stride)
    ref = _brute_force(img, b, stride)
    assert D.shape == ref.shape and len(D) > 0
    np.testing.assert_allclose(D, ref, rtol=1e-10, atol=1e-12)


def test_linear_ramp_closed_form():
    H, W, b = 40, 48, 4
    img = 0.01 * np.arange(W)[None, :] * np.ones((H, 1)) + 0.2
    gx, gy = O.gradients(img)
    np.testing.assert_allclose(gx, 0.01, rtol=1e-12)
    assert np.all(gy == 0)
    D, P = O.descriptors_of_image(img, b, 4)
    ys, xs = O.grid(H, W, b, 4)
    k, checked = 0, 0
    for y0 in ys:
        for x0 in xs:
            # every bin's triangle support (centre +- (b - 1)) inside the image
            if x0 - 1.5 * b - (b - 1) >= 0 and x0 + 1.5 * b + (b - 1) <= W - 1 and \
                    y0 - 1.5 * b - (b - 1) >= 0 and y0 + 1.5 * b + (b - 1) <= H - 1:
                d = D[k].reshape(16, 8)
                np.testing.assert_allclose(d[:, 0], 0.25, rtol=1e-12)
                assert np.all(d[:, 1:] == 0)
                checked += 1
            k += 1
    assert checked >= 4
    assert np.allclose(P[0], (xs[0] / W - 0.5, ys[0] / H - 0.5))


def test_pyramid_and_counts():
    s = O.scales(8, 1)
    assert math.isclose(s[0], math.sqrt(2)) and math.isclose(s[-1], 1 / 8)
    assert all(math.isclose(a / b, math.sqrt(2)) for a, b in zip(s, s[1:]))
    s9 = O.scales(9, 2)
    assert math.isclose(s9[0], 2.0) and math.isclose(s9[-1], 1 / 8)
    assert O.scaled_size(240, 320, 1 / 8) == (30, 40)
    assert O.scaled_size(33, 21, 0.5) == (17, 11)      # halves round up
    ramp = np.arange(20.0)[None, :] * np.ones((12, 1))
    r = O.resize(ramp, 1.0)
    assert np.array_equal(r, ramp)
    r2 = O.resize(ramp, 0.5)
    np.testing.assert_allclose(r2[0, 1:-1], (np.arange(1, 9) + 0.5) * 2 - 0.5, rtol=1e-12)
    assert O.count(240, 320) == 17124
