"""Pins of the FP64 oracle against facts fixed outside the oracle itself.

Each test checks one step of Algorithm 1 (paper Sec. 3.1) or of the improved-FV
normalisation (Sec. 4) against mathematics or a library routine, chosen so
that a dropped term, a sign error, a wrong index or a transposed operand in
the oracle fails at least one of them:

* posteriors (steps 2-3): normalisation, a library Gaussian-mixture model and
  an independent log-density routine;
* U and V (step 4): the Fisher score, i.e. autograd gradients of the GMM
  log-likelihood with respect to the means and standard deviations;
* scalings (step 5): K = 1 and identical-component closed forms;
* signed square root and L2 (step 6): the three properties that fix it;
* invariances of the whole encoder, hard assignment, the threshold mode and
  the degenerate cases (zero norm, empty input).
"""
import math
from decimal import Decimal, getcontext

import numpy as np
import pytest

import oracle
from paper_1604_03498_gb300 import synth


def _case(K=5, D=4, N=40, seed=3, frac=0.8):
    w, mu, var = synth.make_gmm(K, D, seed=seed)
    X = synth.sample_descriptors(w, mu, var, N, seed=seed, gmm_frac=frac)
    return X.astype(np.float64), w.astype(np.float64), mu.astype(np.float64), var.astype(np.float64)


# --- posteriors ------------------------------------------------------------

def test_posteriors_sum_to_one_and_nonnegative():
    X, w, mu, var = _case(K=16, D=8, N=300)
    g = oracle.encode(X, w, mu, var, want_gamma=True)["gamma"]
    assert g.shape == (300, 16)
    assert np.all(g >= 0)
    np.testing.assert_allclose(g.sum(1), 1.0, rtol=0, atol=1e-14)


def test_posteriors_match_library_mixture_model():
    mix = pytest.importorskip("sklearn.mixture")
    X, w, mu, var = _case(K=7, D=5, N=200, seed=11)
    g = oracle.encode(X, w, mu, var, want_gamma=True)["gamma"]
    gm = mix.GaussianMixture(n_components=7, covariance_type="diag")
    gm.weights_ = w / w.sum()
    gm.means_ = mu
    gm.covariances_ = var
    gm.precisions_cholesky_ = 1.0 / np.sqrt(var)
    ref = gm.predict_proba(X)
    np.testing.assert_allclose(g, ref, rtol=0, atol=1e-12)


def test_posteriors_match_scipy_log_densities():
    from scipy.special import softmax
    from scipy.stats import norm
    X, w, mu, var = _case(K=6, D=3, N=100, seed=5, frac=0.5)
    g = oracle.encode(X, w, mu, var, want_gamma=True)["gamma"]
    logp = np.log(w)[None, :] + norm.logpdf(X[:, None, :], loc=mu[None], scale=np.sqrt(var)[None]).sum(-1)
    np.testing.assert_allclose(g, softmax(logp, axis=1), rtol=0, atol=1e-12)


def test_log_likelihood_matrix_and_row_normaliser_match_scipy():
    """L_ik = log w_k + log N(x_i; mu_k, sigma^2_k) + (D/2) log 2pi and
    lse_i = log sum_k exp(L_ik), against scipy's Gaussian log-density and
    logsumexp (the evidence log p(x_i) up to the common 2pi term)."""
    from scipy.special import logsumexp
    from scipy.stats import norm
    X, w, mu, var = _case(K=9, D=7, N=120, seed=8, frac=0.6)
    D = X.shape[1]
    ref = np.log(w)[None, :] + norm.logpdf(X[:, None, :], loc=mu[None], scale=np.sqrt(var)[None]).sum(-1)
    ref += 0.5 * D * math.log(2 * math.pi)
    L = oracle.log_likelihoods(X, w, mu, var)
    np.testing.assert_allclose(L, ref, rtol=1e-13, atol=1e-11)
    g, lse = oracle.posteriors(X, w, mu, var)
    np.testing.assert_allclose(lse, logsumexp(ref, axis=1), rtol=1e-13, atol=1e-11)
    np.testing.assert_allclose(g, oracle.encode(X, w, mu, var, want_gamma=True)["gamma"], rtol=0, atol=1e-15)


# --- first and second order statistics --------------------------------------

def test_statistics_are_loglikelihood_gradients():
    """U_kd = sigma_kd dL/dmu_kd and V_kd = sigma_kd dL/dsigma_kd, where L is the
    GMM log-likelihood of the descriptor set (the Fisher score the encoding is
    built from). Gradients come from float64 autograd of torch's Normal."""
    torch = pytest.importorskip("torch")
    X, w, mu, var = _case(K=6, D=5, N=150, seed=21, frac=0.7)
    r = oracle.encode(X, w, mu, var, want_stats=True)
    m = torch.tensor(mu, dtype=torch.float64, requires_grad=True)
    s = torch.tensor(np.sqrt(var), dtype=torch.float64, requires_grad=True)
    x = torch.tensor(X, dtype=torch.float64)
    lp = torch.distributions.Normal(m[None], s[None]).log_prob(x[:, None, :]).sum(-1)
    L = torch.logsumexp(lp + torch.log(torch.tensor(w, dtype=torch.float64))[None], dim=1).sum()
    gm, gs = torch.autograd.grad(L, (m, s))
    U_ref = (s * gm).detach().numpy()
    V_ref = (s * gs).detach().numpy()
    scale = max(np.abs(U_ref).max(), np.abs(V_ref).max())
    np.testing.assert_allclose(r["U"], U_ref, rtol=0, atol=1e-11 * scale)
    np.testing.assert_allclose(r["V"], V_ref, rtol=0, atol=1e-11 * scale)
    # S0 (sum of posteriors) is the weight gradient's numerator: it sums to N
    np.testing.assert_allclose(r["S0"].sum(), X.shape[0], rtol=1e-13)


# --- scalings: closed forms --------------------------------------------------

def test_single_component_closed_form():
    """K=1: gamma = 1, so u_d = (mean_d - mu_d)/sigma_d and
    v_d = ((s2_d + (mean_d - mu_d)^2)/sigma_d^2 - 1)/sqrt(2), with s2 the
    biased sample variance."""
    g = np.random.default_rng(0)
    D, N = 6, 500
    X = g.normal(0.3, 1.7, size=(N, D))
    mu = g.normal(size=(1, D))
    var = g.uniform(0.2, 3.0, size=(1, D))
    r = oracle.encode(X, np.array([1.0]), mu, var)
    mean = X.mean(0)
    s2 = X.var(0)
    u = (mean - mu[0]) / np.sqrt(var[0])
    v = ((s2 + (mean - mu[0]) ** 2) / var[0] - 1.0) / math.sqrt(2.0)
    np.testing.assert_allclose(r["fv_raw"][:D], u, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(r["fv_raw"][D:], v, rtol=1e-12, atol=1e-14)


def test_identical_components_closed_form():
    """All components share mu and sigma^2: posteriors equal the priors, so
    u_kd = sqrt(w_k) (mean_d - mu_d)/sigma_d and
    v_kd = sqrt(w_k) (mean_i t_id^2 - 1)/sqrt(2). Pins the w-dependence of
    the 1/(N sqrt(w)) and 1/(N sqrt(2w)) scalings."""
    g = np.random.default_rng(1)
    K, D, N = 5, 4, 120
    w = g.dirichlet(np.ones(K))
    mu1 = g.normal(size=D)
    var1 = g.uniform(0.3, 2.0, size=D)
    X = g.normal(size=(N, D)) * 1.3 + 0.2
    r = oracle.encode(X, w, np.tile(mu1, (K, 1)), np.tile(var1, (K, 1)), want_gamma=True)
    np.testing.assert_allclose(r["gamma"], np.tile(w, (N, 1)), rtol=1e-13)
    t = (X - mu1) / np.sqrt(var1)
    u = np.sqrt(w)[:, None] * t.mean(0)[None]
    v = np.sqrt(w)[:, None] * ((t ** 2).mean(0)[None] - 1.0) / math.sqrt(2.0)
    np.testing.assert_allclose(r["fv_raw"][:K * D].reshape(K, D), u, rtol=1e-11, atol=1e-14)
    np.testing.assert_allclose(r["fv_raw"][K * D:].reshape(K, D), v, rtol=1e-11, atol=1e-14)


# --- normalisation -------------------------------------------------------------

def test_signed_sqrt_l2_properties():
    """Unit norm, sign kept, and z_j^2 proportional to |raw_j|: these three fix
    the signed-square-root-then-L2 map uniquely."""
    X, w, mu, var = _case(K=8, D=6, N=90, seed=7)
    r = oracle.encode(X, w, mu, var)
    z, raw = r["fv"], r["fv_raw"]
    assert abs(np.linalg.norm(z) - 1.0) < 1e-14
    assert np.array_equal(np.sign(z), np.sign(raw))
    nz = np.abs(raw) > 1e-300
    ratio = z[nz] ** 2 / np.abs(raw[nz])
    np.testing.assert_allclose(ratio, 1.0 / np.abs(raw).sum(), rtol=1e-12)


# --- hard assignment -----------------------------------------------------------

def test_hard_assignment_on_near_zero_variance_mean():
    """A descriptor exactly on the mean of a component whose variances are 1e-8
    is assigned to it with posterior 1; every other descriptor gets posterior
    ~0 there, so that component's block is u = 0, v = -1 per dimension
    (before scaling)."""
    X, w, mu, var = _case(K=6, D=8, N=50, seed=9)
    k0 = 2
    var = var.copy()
    var[k0] = 1e-8
    X = X.copy()
    X[17] = mu[k0]
    r = oracle.encode(X, w, mu, var, want_gamma=True, want_stats=True)
    g = r["gamma"]
    assert g[17, k0] >= 1.0 - 1e-12
    others = np.delete(np.arange(50), 17)
    assert np.all(g[others, k0] < 1e-12)
    assert np.all(np.abs(r["U"][k0]) < 1e-9)
    np.testing.assert_allclose(r["V"][k0], -1.0, atol=1e-9)


# --- invariances -------------------------------------------------------------------

def test_descriptor_permutation_and_duplication_invariance():
    X, w, mu, var = _case(K=5, D=4, N=70, seed=13)
    ref = oracle.encode(X, w, mu, var)["fv"]
    perm = np.random.default_rng(2).permutation(70)
    np.testing.assert_allclose(oracle.encode(X[perm], w, mu, var)["fv"], ref, atol=1e-14)
    np.testing.assert_allclose(oracle.encode(np.vstack([X, X]), w, mu, var)["fv"], ref, atol=1e-14)


def test_joint_translation_and_scaling_invariance():
    X, w, mu, var = _case(K=5, D=4, N=70, seed=17)
    ref = oracle.encode(X, w, mu, var)["fv"]
    shift = np.array([0.5, -1.25, 2.0, 0.125])
    np.testing.assert_allclose(oracle.encode(X + shift, w, mu + shift, var)["fv"], ref, atol=1e-12)
    a = 3.0
    np.testing.assert_allclose(oracle.encode(X * a, w, mu * a, var * a * a)["fv"], ref, atol=1e-12)


def test_component_permutation_permutes_blocks():
    K, D = 6, 3
    X, w, mu, var = _case(K=K, D=D, N=60, seed=19)
    ref = oracle.encode(X, w, mu, var)["fv"]
    p = np.array([3, 0, 5, 1, 4, 2])
    out = oracle.encode(X, w[p], mu[p], var[p])["fv"]
    u_ref, v_ref = ref[:K * D].reshape(K, D), ref[K * D:].reshape(K, D)
    np.testing.assert_allclose(out[:K * D].reshape(K, D), u_ref[p], atol=1e-14)
    np.testing.assert_allclose(out[K * D:].reshape(K, D), v_ref[p], atol=1e-14)


def test_partition_invariance_of_statistics():
    """Per-block copies summed afterwards equal the single pass (the
    per-block U/V copies and reduction kernel of the paper's Phase 2)."""
    X, w, mu, var = _case(K=5, D=4, N=90, seed=23)
    full = oracle.encode(X, w, mu, var, want_stats=True)
    parts = [oracle.encode(X[a:b], w, mu, var, want_stats=True) for a, b in ((0, 31), (31, 32), (32, 90))]
    for key in ("U", "V", "S0"):
        np.testing.assert_allclose(sum(p[key] for p in parts), full[key], atol=1e-12)


# --- threshold mode, degenerate cases ------------------------------------------------

def test_threshold_mode_bound_and_extremes():
    X, w, mu, var = _case(K=16, D=8, N=400, seed=29, frac=0.6)
    exact = oracle.encode(X, w, mu, var, want_gamma=True, want_stats=True)
    thr = oracle.encode(X, w, mu, var, tau=1e-6, want_stats=True)
    g = exact["gamma"]
    dropped = np.where(g <= 1e-6, g, 0.0)  # mass the threshold removes
    t = (X[:, None, :] - mu[None]) / np.sqrt(var)[None]
    bound_u = np.einsum("ik,ikd->kd", dropped, np.abs(t))
    bound_v = np.einsum("ik,ikd->kd", dropped, np.abs(t * t - 1))
    assert np.all(np.abs(thr["U"] - exact["U"]) <= bound_u + 1e-12)
    assert np.all(np.abs(thr["V"] - exact["V"]) <= bound_v + 1e-12)
    assert np.abs(thr["fv"] - exact["fv"]).max() < 1e-3
    none = oracle.encode(X, w, mu, var, tau=1.0)  # no posterior exceeds 1
    assert none["status"] == oracle.FVO_OK and np.all(none["fv"] == 0)


def test_zero_norm_case_gives_zeros():
    """K=1, D=1, x = mu +- sigma: t = +-1, so U = V = 0 and the FV is all zero."""
    mu = np.array([[0.75]])
    var = np.array([[0.25]])
    X = np.array([[1.25], [0.25]])
    r = oracle.encode(X, np.array([1.0]), mu, var)
    assert r["status"] == oracle.FVO_OK
    assert np.all(r["fv"] == 0) and np.all(r["fv_raw"] == 0)


def test_empty_input_status():
    _, w, mu, var = _case(K=3, D=2, N=5)
    r = oracle.encode(np.zeros((0, 2)), w, mu, var)
    assert r["status"] == oracle.FVO_EMPTY and np.all(r["fv"] == 0)


# --- tiny inputs against a 50-digit evaluation ----------------------------------

def _decimal_fv(X, w, mu, var):
    getcontext().prec = 50
    N, D = len(X), len(X[0])
    K = len(w)
    D_ = [[Decimal(float(v)) for v in row] for row in X]
    M_ = [[Decimal(float(v)) for v in row] for row in mu]
    S2 = [[Decimal(float(v)) for v in row] for row in var]
    W = [Decimal(float(v)) for v in w]
    U = [[Decimal(0)] * D for _ in range(K)]
    V = [[Decimal(0)] * D for _ in range(K)]
    for i in range(N):
        logp = []
        for k in range(K):
            acc = W[k].ln()
            for d in range(D):
                acc -= S2[k][d].ln() / 2 + (D_[i][d] - M_[k][d]) ** 2 / (2 * S2[k][d])
            logp.append(acc)
        m = max(logp)
        e = [(l - m).exp() for l in logp]
        z = sum(e)
        for k in range(K):
            gk = e[k] / z
            for d in range(D):
                t = (D_[i][d] - M_[k][d]) / S2[k][d].sqrt()
                U[k][d] += gk * t
                V[k][d] += gk * (t * t - 1)
    raw = []
    for k in range(K):
        raw += [U[k][d] / (N * W[k].sqrt()) for d in range(D)]
    for k in range(K):
        raw += [V[k][d] / (N * (2 * W[k]).sqrt()) for d in range(D)]
    zz = [(abs(r).sqrt() if r >= 0 else -abs(r).sqrt()) for r in raw]
    nrm = sum(v * v for v in zz).sqrt()
    return np.array([float(v / nrm) for v in zz])


@pytest.mark.parametrize("N,D,K,seed", [(1, 1, 1, 0), (3, 2, 2, 1), (4, 3, 3, 2), (2, 3, 1, 3)])
def test_tiny_inputs_against_50_digit_evaluation(N, D, K, seed):
    g = np.random.default_rng(100 + seed)
    X = g.normal(size=(N, D))
    w = g.dirichlet(np.ones(K))
    mu = g.normal(size=(K, D))
    var = g.uniform(0.1, 1.0, size=(K, D))
    ref = _decimal_fv(X, w, mu, var)
    np.testing.assert_allclose(oracle.encode(X, w, mu, var)["fv"], ref, rtol=0, atol=1e-12)


# --- stored fixtures -------------------------------------------------------------

def _golden():
    import glob
    import json
    import os
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    return sorted(glob.glob(os.path.join(here, "*.json")))


@pytest.mark.parametrize("path", _golden())
def test_golden_fixture_reproduces(path):
    import json
    doc = json.load(open(path))
    N, D, K = doc["N"], doc["D"], doc["K"]
    X = np.array(doc["X"]).reshape(N, D)
    r = oracle.encode(X, np.array(doc["w"]), np.array(doc["mu"]).reshape(K, D), np.array(doc["var"]).reshape(K, D))
    np.testing.assert_allclose(r["fv"], np.array(doc["fv"]), rtol=0, atol=1e-14)
