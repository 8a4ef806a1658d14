"""FV_PREC_BF16X2: the precision form with the posteriors entering the
statistics GEMM as bf16 hi + lo pairs.

The error of the plain BF16 form is dominated by the bfloat16 rounding of
the posteriors (tests/test_bf16_error_budget.py), and the improved-FV
scaling 1/(N sqrt(w)) magnifies it for a component of very small prior: in
the 64-stream serving workload (K=512, D=64, Dirichlet(1) priors) component
279 has w = 1.6e-8 and a 8891-descriptor frame whose statistics for it
cancel 2400-fold reaches 2.02e-3 with bf16 posteriors. With hi + lo
posteriors the same frame, and every other case here, must stay far inside
2e-3 (the CPU model gives 2.8e-5 for it), and the variant must match the
oracle at the shapes of the plain form (one Y stage at D = 64, two at
D <= 48, 1-4 CTA clusters, ragged tails)."""
import numpy as np
import pytest

from gpu_util import TOL, case, gpu_encode, gpu_encode_batch, max_err, oracle_fv, torch_cuda
from paper_1604_03498_gb300 import fv, synth

pytestmark = pytest.mark.gpu
P = fv.FV_PREC_BF16X2


def _rounded(X):
    return synth.to_bf16_grid(np.ascontiguousarray(X, dtype=np.float32))


@pytest.mark.parametrize("K,D,N,seed", [(64, 64, 1000, 1), (256, 64, 19200, 2), (130, 17, 333, 3),
                                         (512, 64, 2000, 4), (384, 48, 3001, 5), (1, 16, 5, 6)])
def test_bf16x2_matches_oracle(K, D, N, seed):
    X, w, mu, var = case(K, D, N, seed)
    st, out = gpu_encode(P, X, w, mu, var)
    assert st == fv.FV_OK
    err = max_err(out, oracle_fv(_rounded(X), w, mu, var))
    assert err <= TOL[P] / 10, err


def test_bf16x2_fixes_the_served_frame_with_a_tiny_prior():
    K, D = 512, 64
    w, mu, var = synth.make_gmm(K, D, seed=1)
    arr = synth.arrival_times(64, 30.0, 60.0, 0.005, seed=5)
    sizes = synth.frame_sizes(len(arr), 8000, 40000, seed=5)
    i = 68275
    s, f, n = int(arr[i][1]), int(arr[i][2]), int(sizes[i])
    X = synth.sample_descriptors(w, mu, var, 40000, seed=90000 + (s * 7 + f) % 32, gmm_frac=0.8)[:n]
    ref = oracle_fv(_rounded(X), w, mu, var)
    _, plain = gpu_encode(fv.FV_PREC_BF16, X, w, mu, var)
    st, fine = gpu_encode(P, X, w, mu, var)
    assert st == fv.FV_OK
    e_plain, e_fine = max_err(plain, ref), max_err(fine, ref)
    assert e_fine <= 2e-4 and e_fine < e_plain / 10, (e_plain, e_fine)


def test_bf16x2_batch_matches_single_frames_and_repeats_bitwise():
    torch = torch_cuda()
    K, D = 512, 64
    _, w, mu, var = case(K, D, 10, 7)
    frames = [synth.sample_descriptors(w, mu, var, n, seed=700 + i, gmm_frac=0.8)
              for i, n in enumerate([5000, 1, 0, 129, 12000])]
    st, outs = gpu_encode_batch(P, frames, w, mu, var)
    assert st == fv.FV_OK
    for fr, o in zip(frames, outs):
        if fr.shape[0] == 0:
            assert np.all(o == 0)
            continue
        _, single = gpu_encode(P, fr, w, mu, var)
        assert max_err(o, single) <= 1e-5
        assert max_err(o, oracle_fv(_rounded(fr), w, mu, var)) <= TOL[P] / 10
    g = fv.fv_gmm_load(w, mu, var, P)
    X = torch.from_numpy(np.concatenate([f for f in frames if len(f)])).cuda().to(torch.bfloat16)
    offs = [0, 5000, 5001, 5130, 17130]
    a = torch.zeros(4, 2 * K * D, device="cuda")
    fv.fv_encode_batch_bf16(g, X, D, offs, a)
    torch.cuda.synchronize()
    ref = a.clone()
    for _ in range(5):
        fv.fv_encode_batch_bf16(g, X, D, offs, a)
        torch.cuda.synchronize()
        assert torch.equal(a, ref)
    g.close()


def test_bf16x2_limits_and_early_termination():
    assert fv.fv_limits(P) == (512, 64)
    _, w, mu, var = case(16, 80, 10, 8)
    with pytest.raises(fv.FVError) as e:
        fv.fv_gmm_load(w, mu, var, P)
    assert e.value.status == fv.FV_ERR_UNSUPPORTED
    torch = torch_cuda()
    import oracle
    X, w, mu, var = case(256, 64, 5000, 9)
    g = fv.fv_gmm_load(w, mu, var, P)
    out = torch.zeros(1, 2 * 256 * 64, device="cuda")
    fv.fv_encode_batch_opts(g, torch.from_numpy(X).cuda(), [0, 5000], out, tau=1e-6)
    torch.cuda.synchronize()
    g.close()
    ref = oracle.encode(_rounded(X), w, mu, var, tau=1e-6)["fv"]
    assert max_err(out.cpu().numpy()[0], ref) <= TOL[P] / 10
