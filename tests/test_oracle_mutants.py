"""Planted mistakes in copies of the FP64 oracle must each fail a pin.

Every mutant below is a plausible slip in one step of the encoder (a dropped
term, a sign, a wrong index, a transposed scaling). A copy of
oracle/fv_oracle.c with the slip is compiled on the CPU and run through the
same checks the oracle pins use (posteriors against scipy, U and V against
autograd gradients of the log-likelihood, the K = 1 and identical-component
closed forms, the signed square root + L2 properties); the unmodified
oracle must pass all of them and every mutant must fail at least one."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1604_03498_gb300 import synth

SRC = os.path.join(os.path.dirname(oracle.__file__), "fv_oracle.c")

MUTANTS = {
    "V without the -1": ("v_k[d] += g * (t * t - 1.0);", "v_k[d] += g * (t * t);"),
    "sqrt(2w) -> sqrt(w)": ("sqrt(2.0 * w[k])", "sqrt(w[k])"),
    "sign of sum log var": ("cst[k] = log(w[k]) - 0.5 * slog;", "cst[k] = log(w[k]) + 0.5 * slog;"),
    "half of the distance dropped": ("L[i * K + k] = cst[k] - 0.5 * q;", "L[i * K + k] = cst[k] - q;"),
    "1/var for 1/sigma": ("isd[d] = 1.0 / sqrt(var[(int64_t)k * D + d]);", "isd[d] = 1.0 / var[(int64_t)k * D + d];"),
    "1/w for 1/sqrt(w)": ("((double)N * sqrt(w[k]))", "((double)N * w[k])"),
    "posteriors not normalised": ("gamma[i * K + k] = exp(l[k] - lse);", "gamma[i * K + k] = exp(l[k] - m);"),
    "signed sqrt loses the sign": ("(a < 0 ? -sqrt(-a) : 0.0)", "(a < 0 ? sqrt(-a) : 0.0)"),
    "wrong mean index": ("const double r = X[i * D + d] - mu[(int64_t)k * D + d];",
                         "const double r = X[i * D + d] - mu[(int64_t)k * D + (D - 1 - d)];"),
    "norm not square-rooted": ("for (int64_t j = 0; j < 2 * KD; ++j) fv[j] /= nrm;",
                               "for (int64_t j = 0; j < 2 * KD; ++j) fv[j] /= nrm2;"),
    "prior dropped": ("cst[k] = log(w[k]) - 0.5 * slog;", "cst[k] = -0.5 * slog;"),
}


def _case(K, D, N, seed, frac=0.7):
    w, mu, var = synth.make_gmm(K, D, seed=seed)
    X = synth.sample_descriptors(w, mu, var, N, seed=seed, gmm_frac=frac)
    return X.astype(np.float64), w.astype(np.float64), mu.astype(np.float64), var.astype(np.float64)


def _failures(lib):
    """Names of the pin checks that the library fails."""
    from scipy.special import softmax
    from scipy.stats import norm
    torch = pytest.importorskip("torch")
    bad = []
    X, w, mu, var = _case(6, 5, 150, 21)
    r = oracle.encode(X, w, mu, var, want_gamma=True, want_stats=True, lib=lib)
    logp = np.log(w)[None] + norm.logpdf(X[:, None, :], loc=mu[None], scale=np.sqrt(var)[None]).sum(-1)
    if not np.allclose(r["gamma"], softmax(logp, axis=1), rtol=0, atol=1e-12):
        bad.append("posteriors")
    m = torch.tensor(mu, requires_grad=True)
    s = torch.tensor(np.sqrt(var), requires_grad=True)
    lp = torch.distributions.Normal(m[None], s[None]).log_prob(torch.tensor(X)[:, None, :]).sum(-1)
    L = torch.logsumexp(lp + torch.log(torch.tensor(w))[None], dim=1).sum()
    gm, gs = torch.autograd.grad(L, (m, s))
    sc = float(max(gm.abs().max(), gs.abs().max())) + 1.0
    if not (np.allclose(r["U"], (s * gm).detach().numpy(), rtol=0, atol=1e-10 * sc)
            and np.allclose(r["V"], (s * gs).detach().numpy(), rtol=0, atol=1e-10 * sc)):
        bad.append("fisher score")
    # K = 1 closed form
    g = np.random.default_rng(0)
    Xk = g.normal(0.3, 1.7, size=(300, 4))
    mk = g.normal(size=(1, 4))
    vk = g.uniform(0.2, 3.0, size=(1, 4))
    rk = oracle.encode(Xk, np.array([1.0]), mk, vk, lib=lib)
    u = (Xk.mean(0) - mk[0]) / np.sqrt(vk[0])
    v = ((Xk.var(0) + (Xk.mean(0) - mk[0]) ** 2) / vk[0] - 1.0) / math.sqrt(2.0)
    if not np.allclose(rk["fv_raw"], np.concatenate([u, v]), rtol=1e-10, atol=1e-12):
        bad.append("K=1 closed form")
    # identical components: posteriors = priors
    K = 4
    wi = g.dirichlet(np.ones(K))
    m1, v1 = g.normal(size=3), g.uniform(0.3, 2.0, size=3)
    Xi = g.normal(size=(80, 3))
    ri = oracle.encode(Xi, wi, np.tile(m1, (K, 1)), np.tile(v1, (K, 1)), lib=lib)
    t = (Xi - m1) / np.sqrt(v1)
    ui = np.sqrt(wi)[:, None] * t.mean(0)[None]
    vi = np.sqrt(wi)[:, None] * ((t ** 2).mean(0) - 1.0)[None] / math.sqrt(2.0)
    if not np.allclose(ri["fv_raw"], np.concatenate([ui.ravel(), vi.ravel()]), rtol=1e-10, atol=1e-12):
        bad.append("identical components")
    # signed square root and L2 fix the normalised vector from the raw one
    raw = r["fv_raw"]
    z = np.sign(raw) * np.sqrt(np.abs(raw))
    if not np.allclose(r["fv"], z / np.linalg.norm(z), rtol=0, atol=1e-14):
        bad.append("signed sqrt + L2")
    return bad


def test_unmodified_oracle_passes_every_check():
    assert _failures(None) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name!r} not found once in the oracle"
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    lib = oracle.load_variant(str(path), str(tmp_path))
    assert _failures(lib), f"no pin caught the planted mistake {name!r}"
