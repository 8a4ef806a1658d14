"""The PCA + position prologue (Sec. 3.1, D = m + 2) on the GPU against the
oracle's FP64 projection, and the whole raw-descriptor encode against the
oracle's projection followed by the oracle's encoder.

Projection: the FP32 kernel agrees with the FP64 projection to FP32
rounding of 128-term dot products (1e-6 absolute on values of order 0.1-1);
the tcgen05 kernel's bfloat16 rows are one rounding (2^-9 relative) of a
projection whose split products err by about 2^-16 of the sum of the
absolute terms sum_k |x_k - mean_k| |P_jk|. Encodes: 1e-4 (FP32 form) and 2e-3 (BF16 form, the oracle
given the exact projection rounded to bfloat16) max-abs on the normalised
vector. Shapes: m = 62 and 78 (D = 64 and 80, the encoder's sizes), m = 48
(the positions land past the padded projection columns), no positions,
ragged row counts (one partial tile, a single row), input widths 16, 64, 128 (tiles landed by one bulk copy)
and 256 (rows loaded by the threads), host and device inputs."""
import numpy as np
import pytest

import oracle
from gpu_util import TOL, max_err, torch_cuda
from paper_1604_03498_gb300 import fv, synth

pytestmark = pytest.mark.gpu


def _inputs(N, m, seed, with_xy=True, Din=128):
    X = synth.sample_sift_like(N, Din, seed=seed)
    P, mean = synth.make_pca(Din, m, seed=seed)
    xy = synth.sample_positions(N, seed=seed) if with_xy else None
    return X, P, mean, xy


@pytest.mark.parametrize("N,m,with_xy,Din", [(1000, 62, True, 128), (333, 78, True, 128), (129, 48, True, 128),
                                             (500, 30, False, 128), (300, 14, True, 16), (385, 40, True, 64),
                                             (257, 62, True, 256), (77, 62, True, 128), (1, 62, True, 128)])
def test_projection_fp32_and_bf16_match_the_oracle(N, m, with_xy, Din):
    torch = torch_cuda()
    X, P, mean, xy = _inputs(N, m, 91, with_xy, Din)
    ref = oracle.pca_project(X, P, mean, xy)
    D = ref.shape[1]
    p = fv.fv_pca_load(P, mean)
    Xd = torch.from_numpy(X).cuda()
    xyd = torch.from_numpy(xy).cuda() if with_xy else None
    y32 = torch.full((N, D), float("nan"), device="cuda")
    fv.fv_pca_project(p, Xd, xyd, y32, False)
    ld = (D + 15) // 16 * 16
    yb = torch.full((N, ld), float("nan"), device="cuda").to(torch.bfloat16)
    fv.fv_pca_project(p, Xd, xyd, yb, True, ld)
    torch.cuda.synchronize()
    p.close()
    a = y32.cpu().numpy().astype(np.float64)
    assert np.abs(a - ref).max() <= 1e-6
    b = yb.float().cpu().numpy().astype(np.float64)
    # one bf16 rounding (2^-9 relative, 2^-8 with margin) of a projection whose split
    # products err by about 2^-16 of the sum of |terms| (2^-14 with margin)
    terms = np.abs(X.astype(np.float64) - mean) @ np.abs(P.astype(np.float64)).T
    bound = 2.0 ** -8 * np.abs(ref[:, :m]) + 2.0 ** -14 * terms
    assert np.all(np.abs(b[:, :m] - ref[:, :m]) <= bound)
    assert np.all(b[:, D:] == 0)
    if with_xy:
        assert np.array_equal(b[:, m:m + 2], synth.to_bf16_grid(xy).astype(np.float64))


@pytest.mark.parametrize("prec,K,m,N,seed", [
    (fv.FV_PREC_FP32, 256, 62, 19200, 92),
    (fv.FV_PREC_BF16, 256, 62, 19200, 93),
    (fv.FV_PREC_BF16, 512, 78, 5000, 94),
    (fv.FV_PREC_FP32, 64, 48, 777, 95),
    (fv.FV_PREC_BF16, 64, 48, 777, 96),
])
def test_encode_raw_descriptors_matches_oracle(prec, K, m, N, seed):
    torch = torch_cuda()
    X, P, mean, xy = _inputs(N, m, seed)
    Y = oracle.pca_project(X, P, mean, xy)
    D = Y.shape[1]
    w, mu, var = synth.make_gmm(K, D, seed=seed)
    mu = (0.3 * mu).astype(np.float32)        # means on the scale of projected SIFT descriptors
    var = (0.05 * var).astype(np.float32)
    g = fv.fv_gmm_load(w, mu, var, prec)
    p = fv.fv_pca_load(P, mean)
    out = torch.full((1, 2 * K * D), float("nan"), device="cuda")
    assert fv.fv_encode_pca(g, p, torch.from_numpy(X).cuda(), torch.from_numpy(xy).cuda(), [0, N], out) == fv.FV_OK
    torch.cuda.synchronize()
    got = out.cpu().numpy()[0]
    Yin = Y if prec == fv.FV_PREC_FP32 else synth.to_bf16_grid(Y.astype(np.float32))
    ref = oracle.encode(Yin, w, mu, var)["fv"]
    assert max_err(got, ref) <= TOL[prec]
    g.close()
    p.close()


def test_encode_raw_descriptors_host_batch_equals_device():
    torch = torch_cuda()
    N1, N2, m, K = 700, 1300, 62, 128
    X, P, mean, xy = _inputs(N1 + N2, m, 97)
    w, mu, var = synth.make_gmm(K, m + 2, seed=97)
    g = fv.fv_gmm_load(w, 0.3 * mu, 0.05 * var, fv.FV_PREC_FP32)
    p = fv.fv_pca_load(P, mean)
    offs = [0, N1, N1 + N2]
    host = np.full((2, 2 * K * (m + 2)), np.nan, np.float32)
    fv.fv_encode_pca(g, p, X, xy, offs, host)
    dev = torch.zeros(2, 2 * K * (m + 2), device="cuda")
    fv.fv_encode_pca(g, p, torch.from_numpy(X).cuda(), torch.from_numpy(xy).cuda(), offs, dev)
    torch.cuda.synchronize()
    assert np.array_equal(host, dev.cpu().numpy())
    Y = oracle.pca_project(X, P, mean, xy)
    for f in range(2):
        ref = oracle.encode(Y[offs[f]:offs[f + 1]], w, 0.3 * mu.astype(np.float64), 0.05 * var.astype(np.float64))
        assert max_err(host[f], ref["fv"]) <= TOL[fv.FV_PREC_FP32]
    g.close()
    p.close()


def test_pca_argument_checks():
    P, mean = synth.make_pca(128, 62, seed=98)
    with pytest.raises(fv.FVError) as e:
        fv.fv_pca_load(np.zeros((79, 128), np.float32))
    assert e.value.status == fv.FV_ERR_UNSUPPORTED
    with pytest.raises(fv.FVError) as e:
        fv.fv_pca_load(np.zeros((10, 100), np.float32))
    assert e.value.status == fv.FV_ERR_UNSUPPORTED
    torch = torch_cuda()
    w, mu, var = synth.make_gmm(16, 60, seed=98)
    g = fv.fv_gmm_load(w, mu, var, fv.FV_PREC_FP32)
    p = fv.fv_pca_load(P, mean)
    with pytest.raises(fv.FVError) as e:   # D must be m + 2
        fv.fv_encode_pca(g, p, torch.zeros(10, 128, device="cuda"), torch.zeros(10, 2, device="cuda"), [0, 10],
                         torch.zeros(1, 2 * 16 * 60, device="cuda"))
    assert e.value.status == fv.FV_ERR_INVALID
    g.close()
    p.close()
