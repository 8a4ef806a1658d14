"""The once-per-GMM preparation (FP64 on the device): the per-component
constants the loader computed must equal the oracle's step-1 constant of
Algorithm 1 (log prior plus Gaussian normaliser) to 1e-12 relative, and the
expanded form used by the BF16 GEMM must equal it minus the mu^2/sigma^2 sum.
Covers padded K and D (K = 300 pads to 320 / 384, D = 80 to 80 / 80) and a
GMM with a near-zero variance."""
import numpy as np
import pytest

import oracle
from gpu_util import case, torch_cuda
from paper_1604_03498_gb300 import fv

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.max(np.abs(a - b) / np.maximum(1.0, np.abs(b))))


@pytest.mark.parametrize("prec", [fv.FV_PREC_FP32, fv.FV_PREC_BF16])
@pytest.mark.parametrize("K,D,tiny", [(300, 80, False), (64, 17, True)])
def test_device_fp64_constants_match_oracle(prec, K, D, tiny):
    torch_cuda()
    _, w, mu, var = case(K, D, 10, 40 + K)
    if tiny:
        var = var.copy()
        var[5] = 1e-8
    g = fv.fv_gmm_load(w, mu, var, prec)
    c_direct, c_expanded = fv.fv_gmm_constants(g)
    g.close()
    w64 = w.astype(np.float64) / np.sum(w.astype(np.float64))   # the loader renormalises the priors
    ref = oracle.log_constants(w64, var)
    quad = np.sum(mu.astype(np.float64) ** 2 / var.astype(np.float64), axis=1)
    assert _rel(c_direct, ref) <= 1e-12
    assert _rel(c_expanded, ref - 0.5 * quad) <= 1e-12
