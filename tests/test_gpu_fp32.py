"""Parity of the plain FP32 form (SIMT kernels) with the FP64 oracle.

Tolerance: 1e-4 max-abs on the normalised Fisher vector. Cases span several
64-row posterior blocks and statistics ranges with ragged tails, padded
component counts (K not a multiple of 64), odd dimensions, the degenerate
shapes (N = 1, K = 1, D = 1, zero norm, N = 0) and the full-size
320x240-frame workload (N=19200, D=64, K=256)."""
import json
import os

import numpy as np
import pytest

from gpu_util import TOL, case, gpu_encode, gpu_encode_batch, max_err, oracle_fv
from paper_1604_03498_gb300 import fv

pytestmark = pytest.mark.gpu
P = fv.FV_PREC_FP32


@pytest.mark.parametrize("K,D,N,seed", [
    (64, 64, 4096, 1),      # single image workload
    (64, 64, 1000, 2),      # ragged tail
    (130, 17, 333, 3),      # padded K, odd D
    (7, 5, 70, 4),
    (256, 80, 777, 5),
    (33, 130, 200, 6),      # D spans three statistics dimension chunks
    (512, 64, 2000, 7),     # Kp=512: the largest row block (64 x 512 log-likelihoods in shared memory)
    (500, 37, 1111, 8),     # K padded to 512, D not a multiple of 16, ragged tail
])
def test_fp32_matches_oracle(K, D, N, seed):
    X, w, mu, var = case(K, D, N, seed)
    st, out = gpu_encode(P, X, w, mu, var)
    assert st == fv.FV_OK
    assert max_err(out, oracle_fv(X, w, mu, var)) <= TOL[P]


def test_fp32_full_frame_320x240():
    X, w, mu, var = case(256, 64, 19200, 11)
    st, out = gpu_encode(P, X, w, mu, var)
    assert st == fv.FV_OK
    err = max_err(out, oracle_fv(X, w, mu, var))
    assert err <= TOL[P], err
    assert abs(np.linalg.norm(out.astype(np.float64)) - 1.0) < 1e-5


@pytest.mark.parametrize("K,D,N,seed", [
    (512, 80, 19200, 17),   # the precision-form comparison shape (320x240 frame, D=80, K=512)
    (512, 64, 40000, 18),   # the largest serving frame (K=512 GMM, N=40000)
])
def test_fp32_full_size_k512(K, D, N, seed):
    X, w, mu, var = case(K, D, N, seed)
    st, out = gpu_encode(P, X, w, mu, var)
    assert st == fv.FV_OK
    err = max_err(out, oracle_fv(X, w, mu, var))
    assert err <= TOL[P], err
    assert abs(np.linalg.norm(out.astype(np.float64)) - 1.0) < 1e-5


def test_fp32_host_buffers_match_device_buffers():
    X, w, mu, var = case(64, 32, 500, 12)
    _, a = gpu_encode(P, X, w, mu, var, on_device=True)
    st, b = gpu_encode(P, X, w, mu, var, on_device=False)
    assert st == fv.FV_OK
    assert np.array_equal(a, b)


@pytest.mark.parametrize("K,D,N", [(1, 1, 1), (1, 8, 5), (5, 1, 9), (64, 64, 1)])
def test_fp32_degenerate_shapes(K, D, N):
    X, w, mu, var = case(K, D, N, 13)
    st, out = gpu_encode(P, X, w, mu, var)
    assert st == fv.FV_OK
    assert max_err(out, oracle_fv(X, w, mu, var)) <= TOL[P]


def test_fp32_zero_norm_gives_zeros():
    mu = np.array([[0.75]], np.float32)
    var = np.array([[0.25]], np.float32)
    X = np.array([[1.25], [0.25]], np.float32)
    st, out = gpu_encode(P, X, np.array([1.0], np.float32), mu, var)
    assert st == fv.FV_OK
    assert np.all(out == 0)


def test_fp32_empty_input():
    _, w, mu, var = case(8, 4, 10, 14)
    st, out = gpu_encode(P, np.zeros((0, 4), np.float32), w, mu, var)
    assert st == fv.FV_ERR_EMPTY
    assert np.all(out == 0)


def test_fp32_hard_assignment_near_zero_variance():
    X, w, mu, var = case(16, 8, 300, 15)
    var = var.copy()
    var[3] = 1e-8
    X = X.copy()
    X[123] = mu[3]
    st, out = gpu_encode(P, X, w, mu, var)
    assert st == fv.FV_OK
    assert max_err(out, oracle_fv(X, w, mu, var)) <= TOL[P]


def test_fp32_batch_equals_single_frames_bitwise():
    """A frame's vector is the same alone and inside a batch (fixed-order
    reductions), including an empty frame in the middle."""
    K, D = 64, 32
    _, w, mu, var = case(K, D, 10, 16)
    from paper_1604_03498_gb300 import synth
    frames = [synth.sample_descriptors(w, mu, var, n, seed=100 + i, gmm_frac=0.8)
              for i, n in enumerate([300, 1, 0, 2049, 64])]
    st, outs = gpu_encode_batch(P, frames, w, mu, var)
    assert st == fv.FV_OK
    for f, o in zip(frames, outs):
        if f.shape[0] == 0:
            assert np.all(o == 0)
            continue
        _, single = gpu_encode(P, f, w, mu, var)
        assert np.array_equal(o, single)
        assert max_err(o, oracle_fv(f, w, mu, var)) <= TOL[P]


def test_fp32_stale_posterior_scratch_is_never_read():
    """The posteriors kernel writes only the 16-component groups that hold a
    non-zero posterior (and a group mask per row); the statistics kernel
    zero-fills the others. A frame encoded after a frame whose posteriors
    were all non-zero (so the reused scratch holds non-zero values where the
    second frame has exact zeros) gives bitwise the same vector as before."""
    K, D, N = 64, 32, 3000
    X, w, mu, var = case(K, D, N, 19)
    a_st, a = gpu_encode(P, X, w, mu, var)
    dense_var = var * 400.0   # every component overlaps every descriptor
    Xd_, _, _, _ = case(K, D, N, 20)
    gpu_encode(P, Xd_, w, mu, dense_var)
    b_st, b = gpu_encode(P, X, w, mu, var)
    assert a_st == b_st == fv.FV_OK
    assert np.array_equal(a, b)
    assert max_err(b, oracle_fv(X, w, mu, var)) <= TOL[P]


def _golden():
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    return sorted(os.path.join(here, f) for f in os.listdir(here) if f.endswith(".json"))


@pytest.mark.parametrize("path", _golden())
def test_fp32_golden_fixtures(path):
    doc = json.load(open(path))
    N, D, K = doc["N"], doc["D"], doc["K"]
    X = np.array(doc["X"], np.float32).reshape(N, D)
    w = np.array(doc["w"], np.float32)
    mu = np.array(doc["mu"], np.float32).reshape(K, D)
    var = np.array(doc["var"], np.float32).reshape(K, D)
    st, out = gpu_encode(P, X, w, mu, var)
    assert st == fv.FV_OK
    assert max_err(out, np.array(doc["fv"])) <= TOL[P]
