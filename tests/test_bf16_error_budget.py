"""Error budget of the BF16 precision form, measured on the CPU.

The CPU model of the form's arithmetic (tests/bf16_emulation.py) is run on a
320x240-shaped frame (N=19200, D=64, K=256) and on the smallest served frame
shape (N=8000, D=64, K=512), each against the FP64 oracle on the same
bf16-rounded descriptors, with every split term in turn removed:

  x*Q_lo, x^2_hi*R_lo, x^2_lo*R_hi  (products of the log-likelihood GEMM),
  X^2_lo                            (plane of the statistics GEMM),

and with the posteriors kept exact instead of rounded to bfloat16. Measured
(max-abs on the normalised vector; tolerance 2e-3):

  case                 kernel   exact-gamma  -xQlo    -x2hiRlo -x2loRhi -X2lo
  N=19200 D=64 K=256   1.4e-4   5.6e-6       9.7e-4   1.6e-3   9.2e-4   1.9e-3
  N=8000  D=64 K=512   2.6e-4   5.1e-5       1.1e-3   1.2e-3   9.4e-4   7.6e-4

Every split term is needed to keep a margin under 2e-3 (dropping any one
multiplies the error by 3 to 13 and uses 38-93% of the budget), and the
remaining error is the bfloat16 rounding of the posteriors before the
statistics GEMM. The GPU tests check that the kernel's output follows this
model (tests/test_gpu_bf16.py)."""
import numpy as np
import pytest

import bf16_emulation as E
import oracle
from paper_1604_03498_gb300 import synth

TOL = 2e-3
TERMS = ("xQlo", "x2hiRlo", "x2loRhi", "X2lo")


@pytest.fixture(scope="module", params=[(256, 64, 19200, 11), (512, 64, 8000, 13)],
                ids=["frame_K256", "served_K512_N8000"])
def budget(request):
    K, D, N, seed = request.param
    w, mu, var = synth.make_gmm(K, D, seed=seed)
    X = synth.to_bf16_grid(synth.sample_descriptors(w, mu, var, N, seed=seed, gmm_frac=0.8)).astype(np.float64)
    ref = oracle.encode(X, w, mu, var)["fv"]

    def err(**kw):
        return float(np.abs(E.encode(X, w, mu, var, **kw) - ref).max())

    out = {"kernel": err(), "exact_gamma": err(gamma="exact"), "hilo_gamma": err(gamma="hilo")}
    for t in TERMS:
        out["-" + t] = err(drop=(t,))
    return out


def test_modelled_kernel_is_inside_the_tolerance_with_margin(budget):
    assert budget["kernel"] <= TOL / 4, budget


@pytest.mark.parametrize("term", TERMS)
def test_every_split_term_is_needed(budget, term):
    assert budget["-" + term] >= 2.5 * budget["kernel"], budget
    assert budget["-" + term] >= 0.3 * TOL, budget


def test_posterior_rounding_dominates_the_remaining_error(budget):
    assert budget["exact_gamma"] <= budget["kernel"] / 4, budget


def test_hi_lo_posteriors_remove_the_posterior_rounding(budget):
    """FV_PREC_BF16X2 keeps the posteriors as bf16 hi + lo in the statistics
    GEMM: its error is that of exact posteriors."""
    assert budget["hilo_gamma"] <= 1.05 * budget["exact_gamma"] + 1e-7, budget
