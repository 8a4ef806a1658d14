"""Dense SIFT oracle: plain, slow, FP64 numpy (test infrastructure only).

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the benchmark's
CPU legs may import it; the product path never does. It shares no code with
the CUDA sources.

The descriptor step of the paper (Sec. 3.1 overview, Sec. 3.2 "Dense SIFT on
GPU", Sec. 4 experiment settings), stated as the steps below. Where the paper
is silent the reading is written next to the step.

1. Pyramid (Sec. 4: scales from 2 down to 1/8 by factors of sqrt 2; the
   8-scale variant drops the x2 scale): scales s_j = 2^((e - j)/2),
   j = 0..n-1, e = 1 and n = 8 by default (e = 2, n = 9: the 9-scale
   setting). Each scaled image has floor(H s + 1/2) x floor(W s + 1/2) pixels, sampled by
   bilinear interpolation at ((u + 0.5) / s - 0.5, (v + 0.5) / s - 0.5),
   coordinates clamped to the image (reading: the paper only says "image
   resizing").
2. Gradients (Sec. 3.1 "the gradients of the pixels"): central differences
   (I[x+1] - I[x-1]) / 2 inside the image, one-sided differences on its
   border; magnitude m = |g|, angle theta = atan2(gy, gx) in [0, 2 pi).
3. Orientation binning ("the gradients of the pixels fall into 8
   orientation bins"): t = theta / (2 pi / 8); the magnitude is split
   linearly between bins floor(t) and floor(t) + 1 (mod 8).
4. Flat-window spatial binning (Sec. 3.2: flat window, triangular
   convolution kernels, "called only twice (once on each dimension)"): each
   orientation channel is convolved with the separable triangle
   k(d) = 1 - |d| / b, |d| < b (b = the spatial bin size, f = 2b - 1 taps),
   zero outside the image; this oracle convolves every pixel (no skipping).
5. Descriptors (Sec. 3.1: 4 x 4 spatial bins x 8 orientations = 128): on a
   grid of centres (x0, y0) with stride S over the positions whose 4b x 4b
   footprint lies in the image, x0 = 2b + S i <= W - 2b (b even, so bin
   centres fall on pixels; reading: the paper gives S = 4 and no bin size,
   4 is used); bin (bx, by) reads
   the filtered channels at (x0 + (bx - 1.5) b, y0 + (by - 1.5) b); entry
   (by * 4 + bx) * 8 + o.
6. Normalisation (reading: the usual SIFT one, VLFeat's scheme the paper
   follows): L2-normalise, cap entries at 0.2, L2-normalise again; a zero
   descriptor stays zero.
7. Positions (Sec. 3.1 "the normalized X and Y"): (x0 / W_s - 0.5,
   y0 / H_s - 0.5) in the scaled image.
Descriptors of all scales are concatenated in scale order, row-major by
(y0, x0) within a scale.
"""
from __future__ import annotations

import math

import numpy as np


def scales(n_scales: int = 8, top: int = 1):
    """The pyramid's scale factors 2^((top - j)/2), largest first."""
    return [2.0 ** ((top - j) / 2.0) for j in range(n_scales)]


def scaled_size(H: int, W: int, s: float):
    return int(math.floor(H * s + 0.5)), int(math.floor(W * s + 0.5))


def resize(img, s: float):
    """Bilinear resampling of a 2-D image by the factor s (step 1)."""
    img = np.asarray(img, np.float64)
    H, W = img.shape
    Hs, Ws = scaled_size(H, W, s)
    y = np.clip((np.arange(Hs) + 0.5) / s - 0.5, 0.0, H - 1.0)
    x = np.clip((np.arange(Ws) + 0.5) / s - 0.5, 0.0, W - 1.0)
    y0 = np.floor(y).astype(int)
    x0 = np.floor(x).astype(int)
    y1 = np.minimum(y0 + 1, H - 1)
    x1 = np.minimum(x0 + 1, W - 1)
    fy = (y - y0)[:, None]
    fx = (x - x0)[None, :]
    top = (1 - fx) * img[y0][:, x0] + fx * img[y0][:, x1]
    bot = (1 - fx) * img[y1][:, x0] + fx * img[y1][:, x1]
    return (1 - fy) * top + fy * bot


def gradients(img):
    """(gx, gy): central differences inside, one-sided on the border (step 2)."""
    img = np.asarray(img, np.float64)
    gx = np.zeros_like(img)
    gy = np.zeros_like(img)
    if img.shape[1] > 1:
        gx[:, 1:-1] = 0.5 * (img[:, 2:] - img[:, :-2])
        gx[:, 0] = img[:, 1] - img[:, 0]
        gx[:, -1] = img[:, -1] - img[:, -2]
    if img.shape[0] > 1:
        gy[1:-1, :] = 0.5 * (img[2:, :] - img[:-2, :])
        gy[0, :] = img[1, :] - img[0, :]
        gy[-1, :] = img[-1, :] - img[-2, :]
    return gx, gy


def orientation_channels(gx, gy, n_bins: int = 8):
    """[n_bins][H][W]: each pixel's magnitude split between its two nearest
    orientation bins (step 3)."""
    m = np.hypot(gx, gy)
    th = np.arctan2(gy, gx)
    th = np.where(th < 0, th + 2 * math.pi, th)
    t = th / (2 * math.pi / n_bins)
    b0 = np.floor(t).astype(int)
    f = t - b0
    ch = np.zeros((n_bins,) + gx.shape)
    for o in range(n_bins):
        ch[o] += np.where(b0 % n_bins == o, m * (1 - f), 0.0)
        ch[o] += np.where((b0 + 1) % n_bins == o, m * f, 0.0)
    return ch


def triangle(b: int):
    """The 2b - 1 taps of k(d) = 1 - |d| / b."""
    return np.array([1.0 - abs(d) / b for d in range(-(b - 1), b)])


def triangular_filter(ch, b: int):
    """Separable triangular convolution of every channel, zero outside the
    image (step 4): a pass along x, then along y, each the sum of the 2b - 1
    shifted, weighted copies."""
    k = triangle(b)
    n, H, W = ch.shape
    pad = np.zeros((n, H, W + 2 * (b - 1)))
    pad[:, :, b - 1:b - 1 + W] = ch
    tmp = sum(k[i] * pad[:, :, i:i + W] for i in range(2 * b - 1))
    pad = np.zeros((n, H + 2 * (b - 1), W))
    pad[:, b - 1:b - 1 + H, :] = tmp
    return sum(k[i] * pad[:, i:i + H, :] for i in range(2 * b - 1))


def grid(Hs: int, Ws: int, b: int, stride: int):
    """Descriptor centres of one scale (step 5): x0 = 2b + stride i <= Ws - 2b."""
    xs = list(range(2 * b, Ws - 2 * b + 1, stride))
    ys = list(range(2 * b, Hs - 2 * b + 1, stride))
    return ys, xs


def normalise(d):
    """L2, cap at 0.2, L2 (step 6); zero stays zero."""
    n = np.linalg.norm(d)
    if n == 0:
        return d
    d = np.minimum(d / n, 0.2)
    n = np.linalg.norm(d)
    return d / n if n > 0 else d


def descriptors_of_image(img, b: int = 4, stride: int = 4):
    """All descriptors (N x 128) and positions (N x 2) of one (scaled) image."""
    img = np.asarray(img, np.float64)
    Hs, Ws = img.shape
    gx, gy = gradients(img)
    filt = triangular_filter(orientation_channels(gx, gy), b)
    ys, xs = grid(Hs, Ws, b, stride)
    D, P = [], []
    for y0 in ys:
        for x0 in xs:
            d = np.zeros(128)
            for by in range(4):
                for bx in range(4):
                    cy = int(round(y0 + (by - 1.5) * b))
                    cx = int(round(x0 + (bx - 1.5) * b))
                    d[(by * 4 + bx) * 8:(by * 4 + bx) * 8 + 8] = filt[:, cy, cx]
            D.append(normalise(d))
            P.append((x0 / Ws - 0.5, y0 / Hs - 0.5))
    return np.array(D).reshape(-1, 128), np.array(P).reshape(-1, 2)


def dense_sift(img, b: int = 4, stride: int = 4, n_scales: int = 8, top: int = 1):
    """Descriptors and positions of one image over the pyramid (all steps)."""
    Ds, Ps = [], []
    for s in scales(n_scales, top):
        d, p = descriptors_of_image(resize(img, s), b, stride)
        Ds.append(d)
        Ps.append(p)
    return np.concatenate(Ds), np.concatenate(Ps)


def count(H: int, W: int, b: int = 4, stride: int = 4, n_scales: int = 8, top: int = 1) -> int:
    n = 0
    for s in scales(n_scales, top):
        Hs, Ws = scaled_size(H, W, s)
        ys, xs = grid(Hs, Ws, b, stride)
        n += len(ys) * len(xs)
    return n
