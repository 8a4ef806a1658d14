"""Early termination (paper Sec. 3.3, Algorithm 5) on the GPU.

With a posterior threshold tau > 0, fv_encode_batch_opts drops statistics
terms whose posterior is not above tau and skips blocks whose posteriors are
all at or below it (FP32 form: a warp's row of 16 components; BF16 form: a
16-row x 128-component K step of the statistics GEMM). The result must match
the oracle's threshold mode (the same definition in FP64) within the form's
tolerance, stay within the exact encoding's distance to the threshold mode,
and tau = 0 through the options entry must give the exact path's bits."""
import numpy as np
import pytest

from gpu_util import TOL, case, max_err, torch_cuda
import oracle
from paper_1604_03498_gb300 import fv, synth

pytestmark = pytest.mark.gpu
TAU = 1e-6


def _run(prec, X, w, mu, var, tau, offsets=None, bf16_input=False):
    torch = torch_cuda()
    g = fv.fv_gmm_load(w, mu, var, prec)
    K, D = mu.shape
    offs = offsets if offsets is not None else [0, X.shape[0]]
    B = len(offs) - 1
    Xd = torch.from_numpy(np.ascontiguousarray(X, np.float32)).cuda()
    if bf16_input:
        Xd = Xd.to(torch.bfloat16)
    out = torch.full((B, 2 * K * D), float("nan"), device="cuda")
    cnt = torch.zeros(2, dtype=torch.int64, device="cuda")
    st = fv.fv_encode_batch_opts(g, Xd, offs, out, tau=tau, skip_counts=cnt)
    torch.cuda.synchronize()
    g.close()
    return st, out.cpu().numpy(), [int(v) for v in cnt.cpu()]


def _ref(X, w, mu, var, tau):
    return oracle.encode(X, w, mu, var, tau=tau)["fv"]


@pytest.mark.parametrize("K,D,N,seed", [(256, 64, 19200, 61), (64, 64, 4096, 62), (130, 17, 777, 63)])
def test_fp32_threshold_mode_matches_oracle(K, D, N, seed):
    X, w, mu, var = case(K, D, N, seed)
    st, out, (skipped, visited) = _run(fv.FV_PREC_FP32, X, w, mu, var, TAU)
    assert st == fv.FV_OK
    thr, exact = _ref(X, w, mu, var, TAU), _ref(X, w, mu, var, 0.0)
    assert max_err(out[0], thr) <= TOL[fv.FV_PREC_FP32]
    assert max_err(out[0], exact) <= max_err(thr, exact) + TOL[fv.FV_PREC_FP32]
    assert 0 < skipped <= visited
    assert visited == N * ((K + 63) // 64 * 64 // 16)


def test_fp32_threshold_zero_is_the_exact_path_bitwise():
    X, w, mu, var = case(256, 64, 5000, 64)
    torch = torch_cuda()
    g = fv.fv_gmm_load(w, mu, var, fv.FV_PREC_FP32)
    a = torch.zeros(1, 2 * 256 * 64, device="cuda")
    b = torch.zeros(1, 2 * 256 * 64, device="cuda")
    Xd = torch.from_numpy(X).cuda()
    fv.fv_encode_batch(g, Xd, [0, 5000], a)
    fv.fv_encode_batch_opts(g, Xd, [0, 5000], b, tau=0.0)
    torch.cuda.synchronize()
    g.close()
    assert torch.equal(a, b)


@pytest.mark.parametrize("K,D,N,seed", [(256, 64, 19200, 65), (512, 80, 3000, 66), (64, 32, 1000, 67)])
def test_bf16_threshold_mode_matches_oracle(K, D, N, seed):
    X, w, mu, var = case(K, D, N, seed)
    Xr = synth.to_bf16_grid(X)
    st, out, (skipped, visited) = _run(fv.FV_PREC_BF16, X, w, mu, var, TAU)
    assert st == fv.FV_OK
    assert max_err(out[0], _ref(Xr, w, mu, var, TAU)) <= TOL[fv.FV_PREC_BF16]
    assert 0 <= skipped <= visited and visited > 0


@pytest.mark.parametrize("prec", [fv.FV_PREC_BF16, fv.FV_PREC_BF16X2])
def test_bf16_block_skips_on_sorted_descriptors_and_all_skipped_units(prec):
    """Descriptors ordered by their generating component put many 16-row K
    steps entirely on one CTA's components, so the other CTA skips them; a
    frame drawn only from components 0-127 (components 128-255 far away)
    leaves the second CTA no posterior above tau in any K step, which must
    still give exact zeros for those components' statistics. Both BF16
    forms (the hi + lo posteriors go through the statistics GEMM in two
    64-row halves)."""
    K, D = 256, 32
    w, mu, var = synth.make_gmm(K, D, seed=68)
    mu = mu.copy()
    mu[128:] += 40.0
    g = np.random.default_rng(68)
    comp = np.sort(g.choice(128, size=6000, p=w[:128] / w[:128].sum()))
    X1 = (mu[comp] + np.sqrt(var[comp]) * g.standard_normal((6000, D))).astype(np.float32)
    comp2 = np.sort(g.choice(K, size=6000, p=w / w.sum()))
    X2 = (mu[comp2] + np.sqrt(var[comp2]) * g.standard_normal((6000, D))).astype(np.float32)
    X = np.concatenate([X1, X2])
    st, out, (skipped, visited) = _run(prec, X, w, mu, var, TAU, offsets=[0, 6000, 12000])
    assert st == fv.FV_OK
    assert skipped > visited // 4, (skipped, visited)
    for f, Xf in enumerate((X1, X2)):
        ref = _ref(synth.to_bf16_grid(Xf), w, mu, var, TAU)
        assert max_err(out[f], ref) <= TOL[prec]
    # the first frame's components 128..255 have no posterior above tau: zero blocks
    KD = K * D
    assert np.all(out[0][128 * D:KD] == 0) and np.all(out[0][KD + 128 * D:] == 0)


def test_bf16_threshold_zero_is_the_exact_path_bitwise():
    torch = torch_cuda()
    X, w, mu, var = case(256, 64, 5000, 69)
    g = fv.fv_gmm_load(w, mu, var, fv.FV_PREC_BF16)
    Xb = torch.from_numpy(X).cuda().to(torch.bfloat16)
    a = torch.zeros(1, 2 * 256 * 64, device="cuda")
    b = torch.zeros(1, 2 * 256 * 64, device="cuda")
    fv.fv_encode_batch_bf16(g, Xb, 64, [0, 5000], a)
    fv.fv_encode_batch_opts(g, Xb, [0, 5000], b, tau=0.0, ld_x=64)
    torch.cuda.synchronize()
    g.close()
    assert torch.equal(a, b)


def test_threshold_outside_its_range_is_rejected():
    torch = torch_cuda()
    X, w, mu, var = case(8, 4, 10, 70)
    g = fv.fv_gmm_load(w, mu, var, fv.FV_PREC_FP32)
    out = torch.zeros(1, 64, device="cuda")
    for tau in (-1e-6, 1.0, float("nan")):
        with pytest.raises(fv.FVError) as e:
            fv.fv_encode_batch_opts(g, torch.from_numpy(X).cuda(), [0, 10], out, tau=tau)
        assert e.value.status == fv.FV_ERR_INVALID
    g.close()
