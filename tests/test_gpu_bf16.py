"""Parity of the BF16 precision form (tcgen05 tensor-core GEMMs with hi+lo
split products) with the FP64 oracle.

The precision form stores descriptors as bfloat16, so the oracle is handed
the same bfloat16-rounded descriptors (both sides encode the identical
input); the tolerance is 2e-3 max-abs on the normalised Fisher vector. The
full-size cases also check the error against the oracle on the original FP32
descriptors (input quantisation included) against the same bound.

Shapes span several 128-row tiles with ragged tails, frame ranges ending
inside a tile, K padded to 128, clusters of 1 to 4 CTAs (128 components
each, posteriors normalised across the cluster), D not a multiple of 16, a
single Y stage (D=80 with K=512), and the degenerate N = 1 / K = 1 cases."""
import numpy as np
import pytest

from gpu_util import TOL, case, gpu_encode, gpu_encode_batch, max_err, oracle_fv, torch_cuda
from paper_1604_03498_gb300 import fv, synth

pytestmark = pytest.mark.gpu
P = fv.FV_PREC_BF16


def _rounded(X):
    return synth.to_bf16_grid(np.ascontiguousarray(X, dtype=np.float32))


@pytest.mark.parametrize("K,D,N,seed", [
    (64, 64, 1000, 1),      # Kp=128: one CTA per cluster
    (256, 64, 777, 2),      # 2-CTA clusters, ragged last tile
    (130, 17, 333, 3),      # padded K and D
    (300, 32, 1290, 4),     # Kp=384: 3-CTA clusters
    (512, 64, 2000, 5),     # 4-CTA clusters
    (256, 80, 513, 6),      # D=80: five 16-column blocks
    (1, 16, 5, 7),
    (64, 64, 1, 8),
])
def test_bf16_matches_oracle(K, D, N, seed):
    X, w, mu, var = case(K, D, N, seed)
    Xr = _rounded(X)
    st, out = gpu_encode(P, X, w, mu, var)
    assert st == fv.FV_OK
    assert np.all(np.isfinite(out))
    err = max_err(out, oracle_fv(Xr, w, mu, var))
    assert err <= TOL[P], err


@pytest.mark.parametrize("K,D", [(256, 64), (512, 80)])
def test_bf16_full_frame_320x240(K, D):
    X, w, mu, var = case(K, D, 19200, 20 + K)
    st, out = gpu_encode(P, X, w, mu, var)
    assert st == fv.FV_OK
    e_same_input = max_err(out, oracle_fv(_rounded(X), w, mu, var))
    e_fp32_input = max_err(out, oracle_fv(X, w, mu, var))
    assert e_same_input <= TOL[P], e_same_input
    assert e_fp32_input <= TOL[P], e_fp32_input


def test_bf16_raw_entry_matches_fp32_input_entry():
    """fv_encode_batch_bf16 on descriptors already stored as bf16 (row pitch
    larger than D) gives the same vectors as the FP32-input call."""
    torch = torch_cuda()
    K, D, N = 256, 64, 3000
    X, w, mu, var = case(K, D, N, 30)
    g = fv.fv_gmm_load(w, mu, var, P)
    ld = 72
    Xb = torch.zeros((N, ld), dtype=torch.bfloat16, device="cuda")
    Xb[:, :D] = torch.from_numpy(X).cuda().to(torch.bfloat16)
    out_raw = torch.zeros(1, 2 * K * D, device="cuda")
    fv.fv_encode_batch_bf16(g, Xb, ld, [0, N], out_raw)
    out_f32 = torch.zeros(2 * K * D, device="cuda")
    fv.fv_encode(g, torch.from_numpy(X).cuda(), out_f32)
    torch.cuda.synchronize()
    g.close()
    assert max_err(out_raw.cpu().numpy()[0], out_f32.cpu().numpy()) <= 1e-6


@pytest.mark.parametrize("K,D", [(256, 64), (512, 80)])
def test_bf16_batch_matches_single_frames(K, D):
    """Frames of mixed sizes in one call: units start and end inside tiles,
    shares hold several units (several statistics write-outs per cluster);
    K=512, D=80 runs 4-CTA clusters with a single Y stage."""
    _, w, mu, var = case(K, D, 10, 31)
    frames = [synth.sample_descriptors(w, mu, var, n, seed=300 + i, gmm_frac=0.8)
              for i, n in enumerate([5000, 1, 0, 129, 12000])]
    st, outs = gpu_encode_batch(P, frames, w, mu, var)
    assert st == fv.FV_OK
    for f, o in zip(frames, outs):
        if f.shape[0] == 0:
            assert np.all(o == 0)
            continue
        _, single = gpu_encode(P, f, w, mu, var)
        assert max_err(o, single) <= 1e-5
        assert max_err(o, oracle_fv(_rounded(f), w, mu, var)) <= TOL[P]


def test_bf16_hard_assignment_near_zero_variance():
    """A bf16-exact descriptor on the mean of a component with variances 1e-8:
    the expanded-form statistics must still centre exactly (hi+lo x^2, FP64
    centring), giving u = 0, v = -beta/N for that component."""
    X, w, mu, var = case(16, 16, 300, 32)
    mu = mu.copy()
    mu[3] = _rounded(mu[3:4])[0]
    var = var.copy()
    var[3] = 1e-8
    X = _rounded(X).copy()
    X[123] = mu[3]
    st, out = gpu_encode(P, X, w, mu, var)
    assert st == fv.FV_OK
    assert max_err(out, oracle_fv(X, w, mu, var)) <= TOL[P]


def test_bf16_empty_input():
    _, w, mu, var = case(64, 16, 10, 33)
    st, out = gpu_encode(P, np.zeros((0, 16), np.float32), w, mu, var)
    assert st == fv.FV_ERR_EMPTY
    assert np.all(out == 0)


@pytest.mark.parametrize("K,D", [(256, 64), (512, 64), (512, 80)])
def test_bf16_repeated_calls_are_bitwise_identical(K, D):
    """Sixteen 320x240-shaped frames in one call, repeated: every repeat gives
    the same bits (the cluster exchanges, the stage and TMEM hand-offs and
    the slot reduction leave no order-dependent result), and frames sampled
    from the batch match the oracle."""
    torch = torch_cuda()
    _, w, mu, var = case(K, D, 10, 34)
    F, N = 16, 19200
    frames = [synth.sample_descriptors(w, mu, var, N, seed=400 + i, gmm_frac=0.8) for i in range(F)]
    g = fv.fv_gmm_load(w, mu, var, P)
    X = torch.from_numpy(np.concatenate(frames)).cuda().to(torch.bfloat16)
    offs = [i * N for i in range(F + 1)]
    out = torch.zeros(F, 2 * K * D, device="cuda")
    fv.fv_encode_batch_bf16(g, X, D, offs, out)
    torch.cuda.synchronize()
    ref = out.clone()
    for _ in range(12):
        fv.fv_encode_batch_bf16(g, X, D, offs, out)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
    g.close()
    got = ref.cpu().numpy()
    for f in (0, F - 1):
        assert max_err(got[f], oracle_fv(_rounded(frames[f]), w, mu, var)) <= TOL[P]


@pytest.mark.parametrize("K,D,N,seed", [(256, 64, 19200, 11), (512, 64, 8000, 13), (512, 64, 11173, 14)])
def test_bf16_kernel_follows_the_cpu_model_of_its_roundings(K, D, N, seed):
    """The fused kernel's output follows the CPU model of the precision
    form's roundings (tests/bf16_emulation.py: bf16 split operands, bf16
    posteriors), so the error budget measured on the CPU
    (tests/test_bf16_error_budget.py) is the kernel's: the two agree to well
    within the tolerance, and both are inside it."""
    import bf16_emulation as E
    X, w, mu, var = case(K, D, N, seed)
    Xr = _rounded(X).astype(np.float64)
    st, out = gpu_encode(P, X, w, mu, var)
    assert st == fv.FV_OK
    model = E.encode(Xr, w, mu, var)
    ref = oracle_fv(Xr, w, mu, var)
    assert max_err(out, model) <= TOL[P] / 4
    assert max_err(out, ref) <= TOL[P]
    assert max_err(model, ref) <= TOL[P]
