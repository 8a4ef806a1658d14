"""Pins of the oracle's EM step for the diagonal GMM (the model Sec. 3.1
assumes trained beforehand), each against something outside the oracle:

* one iteration of scikit-learn's GaussianMixture (diagonal covariances,
  started from the same parameters): new weights, means, variances and the
  log-likelihood lower bound of the E-step;
* the K = 1 closed form: sample mean and biased sample variance;
* EM's monotone log-likelihood over several steps;
* the log-likelihood against scipy's Gaussian log-density."""
import math

import numpy as np
import pytest

import oracle
from paper_1604_03498_gb300 import synth


def _case(K, D, N, seed):
    w, mu, var = synth.make_gmm(K, D, seed=seed)
    X = synth.sample_descriptors(w, mu, var, N, seed=seed, gmm_frac=0.8)
    return X.astype(np.float64), w.astype(np.float64), mu.astype(np.float64), var.astype(np.float64)


def test_em_step_matches_scikit_learn_one_iteration():
    mix = pytest.importorskip("sklearn.mixture")
    X, w, mu, var = _case(6, 5, 400, 71)
    reg = 1e-6
    gm = mix.GaussianMixture(n_components=6, covariance_type="diag", max_iter=1, tol=0.0, reg_covar=reg,
                             weights_init=w / w.sum(), means_init=mu, precisions_init=1.0 / var, random_state=0)
    import warnings
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")   # one iteration does not converge
        gm.fit(X)
    w2, mu2, var2, ll = oracle.em_step(X, w / w.sum(), mu, var, reg=reg)
    np.testing.assert_allclose(w2, gm.weights_, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(mu2, gm.means_, rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(var2, gm.covariances_, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(ll, gm.lower_bound_, rtol=1e-12)


def test_em_step_single_component_closed_form():
    g = np.random.default_rng(3)
    X = g.normal(0.5, 2.0, size=(300, 4))
    w2, mu2, var2, ll = oracle.em_step(X, np.array([1.0]), np.zeros((1, 4)), np.ones((1, 4)), reg=0.0)
    np.testing.assert_allclose(w2, [1.0], rtol=1e-14)
    np.testing.assert_allclose(mu2[0], X.mean(0), rtol=1e-12)
    np.testing.assert_allclose(var2[0], X.var(0), rtol=1e-11)


def test_em_log_likelihood_is_monotone_and_matches_scipy():
    from scipy.special import logsumexp
    from scipy.stats import norm
    X, w, mu, var = _case(5, 3, 500, 72)
    mu = mu + 0.7   # start away from the generating model
    prev = -np.inf
    for _ in range(8):
        w2, mu2, var2, ll = oracle.em_step(X, w, mu, var, reg=1e-9)
        ref = logsumexp(np.log(w)[None] + norm.logpdf(X[:, None, :], mu[None], np.sqrt(var)[None]).sum(-1), axis=1)
        assert math.isclose(ll, ref.mean(), rel_tol=1e-12)
        assert ll >= prev - 1e-12
        prev = ll
        w, mu, var = w2, mu2, var2
