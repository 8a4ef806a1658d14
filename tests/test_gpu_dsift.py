"""Dense SIFT on the GPU against the FP64 oracle (Sec. 3.1-3.2), and images
in / Fisher vectors out against the oracle's dense SIFT, PCA and encoder.

Descriptor tolerance: the kernels work in FP32 (bilinear resampling with
FP32 coordinates, gradient differences, atan2f, 2 x (2b - 1) tap sums, the
two normalisations); every step is continuous in its inputs (the
orientation split and the 0.2 cap included), so the entries, at most about
0.35, agree to a few FP32 rounding steps of the filtered values relative to
the descriptor's norm: 2e-5 absolute is the bound used (measured values are
reported by the assertion message)."""
import numpy as np
import pytest

import oracle
from gpu_util import TOL, max_err, torch_cuda
from oracle import dsift_oracle as O
from paper_1604_03498_gb300 import fv, synth

pytestmark = pytest.mark.gpu
DTOL = 2e-5


def _gpu_dsift(frames, on_device=True, **params):
    torch = torch_cuda()
    B, H, W = frames.shape
    n = fv.fv_dsift_count(H, W, **params)
    desc = torch.full((B, n, 128), float("nan"), device="cuda")
    xy = torch.full((B, n, 2), float("nan"), device="cuda")
    src = torch.from_numpy(frames).cuda() if on_device else frames
    fv.fv_dsift(src, desc, xy, **params)
    torch.cuda.synchronize()
    return desc.cpu().numpy(), xy.cpu().numpy()


@pytest.mark.parametrize("H,W,params,on_device", [
    (240, 320, {}, True),                                     # a 320x240 frame, the paper's 8 scales
    (57, 83, {}, False),                                      # odd sizes, host frames
    (120, 160, dict(bin_size=8, stride=4), True),
    (100, 130, dict(bin_size=4, stride=2, n_scales=9, top_scale=2), True),
    (200, 300, dict(bin_size=16, stride=16), True),           # the widest pixel span of an x-pass block
    (64, 96, dict(bin_size=2, stride=1), True),               # three 64-column segments per row at the top scale
])
def test_descriptors_match_oracle(H, W, params, on_device):
    frames = synth.make_frames(2, H, W, seed=H + W)
    d, p = _gpu_dsift(frames, on_device, **params)
    kw = dict(b=params.get("bin_size", 4), stride=params.get("stride", 4), n_scales=params.get("n_scales", 8),
              top=params.get("top_scale", 1))
    for f in range(2):
        D, P = O.dense_sift(frames[f].astype(np.float64), **kw)
        assert d[f].shape == D.shape
        err = float(np.abs(d[f] - D).max())
        assert err <= DTOL, err
        assert float(np.abs(p[f] - P).max()) <= 1e-6
        nz = np.linalg.norm(D, axis=1) > 0
        np.testing.assert_allclose(np.linalg.norm(d[f][nz], axis=1), 1.0, atol=1e-5)


def test_flat_image_gives_zero_descriptors():
    frames = np.full((1, 64, 64), 0.5, np.float32)
    d, _ = _gpu_dsift(frames)
    assert np.all(d == 0)


@pytest.mark.parametrize("prec", [fv.FV_PREC_FP32, fv.FV_PREC_BF16])
def test_images_to_fisher_vectors_match_oracle(prec):
    torch = torch_cuda()
    B, H, W, m, K = 2, 240, 320, 62, 64
    frames = synth.make_frames(B, H, W, seed=5)
    P, mean = synth.make_pca(128, m, seed=5)
    w, mu, var = synth.make_gmm(K, m + 2, seed=5)
    mu, var = (0.3 * mu).astype(np.float32), (0.05 * var).astype(np.float32)
    g = fv.fv_gmm_load(w, mu, var, prec)
    pca = fv.fv_pca_load(P, mean)
    out = torch.full((B, 2 * K * (m + 2)), float("nan"), device="cuda")
    fv.fv_encode_images(g, pca, torch.from_numpy(frames).cuda(), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for f in range(B):
        D, Pxy = O.dense_sift(frames[f].astype(np.float64))
        Y = oracle.pca_project(D, P, mean, Pxy)
        Yin = Y if prec == fv.FV_PREC_FP32 else synth.to_bf16_grid(Y.astype(np.float32))
        ref = oracle.encode(Yin, w, mu, var)["fv"]
        assert max_err(got[f], ref) <= TOL[prec]
    g.close()
    pca.close()
