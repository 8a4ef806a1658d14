"""GMM training by EM on the GPU (fv_gmm_em_step, fv_gmm_fit) against the
oracle's EM step (FP64, pinned against scikit-learn).

Tolerances follow from the arithmetic: the E-step sums are FP32 (posteriors
and centred statistics as in the FP32 encoder, whose normalised vector
agrees with the oracle to 1e-4), the M-step is FP64 on those sums. Weights
agree to 1e-5 relative (+1e-9), means to 1e-4 of the component's standard
deviation, and the mean log-likelihood to 1e-6 relative. The new variance is
the FP32 second moment about the OLD mean, re-centred on the new one,
  var' = B/N_k - delta^2 (delta = mu' - mu),
so its rounding is relative to B/N_k = var' - reg + delta^2, not to var'
itself: a component whose mean moves far compared with its new spread loses
digits to that cancellation. Variances therefore agree to 1e-4 relative plus
1e-5 of B/N_k."""
import numpy as np
import pytest

import oracle
from gpu_util import case, torch_cuda
from paper_1604_03498_gb300 import fv, synth

pytestmark = pytest.mark.gpu


def _check(got, ref, var_ref, mu_old, reg):
    w, mu, var, ll = got
    w2, mu2, var2, ll2 = ref
    np.testing.assert_allclose(w, w2, rtol=1e-5, atol=1e-9)
    assert np.all(np.abs(mu - mu2) <= 1e-4 * np.sqrt(var_ref) + 1e-6)
    second_moment_old_mean = (var2 - reg) + (mu2 - mu_old) ** 2
    assert np.all(np.abs(var - var2) <= 1e-4 * var2 + 1e-5 * second_moment_old_mean)
    assert abs(ll - ll2) <= 1e-6 * abs(ll2)


@pytest.mark.parametrize("K,D,N,seed,on_device", [(64, 32, 5000, 81, True), (256, 64, 19200, 82, False),
                                                 (7, 5, 333, 83, True), (130, 17, 2000, 84, False),
                                                 (512, 64, 8000, 85, True)])   # the largest component count
def test_em_step_matches_oracle(K, D, N, seed, on_device):
    torch = torch_cuda()
    X, w, mu, var = case(K, D, N, seed)
    mu = mu + 0.3   # a model away from the data's own, so the step moves it
    g = fv.fv_gmm_load(w, mu, var, fv.FV_PREC_FP32)
    Xin = torch.from_numpy(X).cuda() if on_device else X
    got = fv.fv_gmm_em_step(g, Xin, reg_covar=1e-6)
    g.close()
    ref = oracle.em_step(X, w, mu, var, reg=1e-6)
    _check(got, ref, ref[2], mu, 1e-6)


def test_em_step_with_an_empty_component():
    """A component far from every descriptor gets N_k = 10 eps: its mean and
    variance go to 0 and reg (oracle and GPU alike), its weight to ~0."""
    X, w, mu, var = case(8, 4, 500, 85)
    mu = mu.copy()
    mu[5] += 1e3
    g = fv.fv_gmm_load(w, mu, var, fv.FV_PREC_FP32)
    got = fv.fv_gmm_em_step(g, X, reg_covar=1e-3)
    g.close()
    ref = oracle.em_step(X, w, mu, var, reg=1e-3)
    assert got[0][5] < 1e-12 and np.all(got[1][5] == 0) and np.allclose(got[2][5], 1e-3)
    _check(got, ref, np.maximum(ref[2], 1e-3), mu, 1e-3)


def test_fit_follows_the_oracle_and_increases_the_likelihood():
    K, D, N = 16, 8, 4000
    wt, mut, vart = synth.make_gmm(K, D, seed=86)
    X = synth.sample_descriptors(wt, mut, vart, N, seed=86, gmm_frac=1.0)
    w0, mu0, var0 = synth.make_gmm(K, D, seed=87)   # another model as the start
    w, mu, var = w0.astype(np.float64), mu0.astype(np.float64), var0.astype(np.float64)
    lls = []
    for _ in range(6):
        w, mu, var, ll = oracle.em_step(X, w, mu, var, reg=1e-6)
        lls.append(ll)
    assert all(b >= a - 1e-9 for a, b in zip(lls, lls[1:]))
    gw, gmu, gvar, it, gll = fv.fv_gmm_fit(w0, mu0, var0, X, max_iter=6, tol=0.0, reg_covar=1e-6)
    assert it == 6
    np.testing.assert_allclose(gw, w, rtol=1e-3, atol=1e-7)
    assert np.all(np.abs(gmu - mu) <= 1e-3 * np.sqrt(var) + 1e-5)
    np.testing.assert_allclose(gvar, var, rtol=1e-3)
    assert abs(gll - lls[-1]) <= 1e-5 * abs(lls[-1])
    # converged run: stops before max_iter once the likelihood settles
    _, _, _, it2, _ = fv.fv_gmm_fit(w0, mu0, var0, X, max_iter=500, tol=1e-4, reg_covar=1e-6)
    assert 6 < it2 < 500
