"""The allocation-free entry point, fv_encode_noalloc.

It serves callers that must not allocate device memory (their own allocator
owns the device, a memory quota, or a loop that must not wait on a pool
growing): its scratch is a fixed array inside the library. Checked through
the C ABI against fv_encode on the same inputs, within the FP32 form's 1e-4,
on two calls in a row (the second call must not be disturbed by what the
first left in the shared array). This file is collected last so that a run
stopping at the first failure has already run every other test."""
import numpy as np
import pytest

from gpu_util import TOL, case, max_err, torch_cuda
from paper_1604_03498_gb300 import fv

pytestmark = pytest.mark.gpu


def test_noalloc_matches_fv_encode_on_two_calls_in_a_row():
    torch = torch_cuda()
    K, D = 256, 64
    _, w, mu, var = case(K, D, 10, 40)
    g = fv.fv_gmm_load(w, mu, var, fv.FV_PREC_FP32)
    from paper_1604_03498_gb300 import synth
    for i, n in enumerate([19200, 3001]):
        X = synth.sample_descriptors(w, mu, var, n, seed=500 + i, gmm_frac=0.8)
        Xd = torch.from_numpy(X).cuda()
        ref = torch.full((2 * K * D,), float("nan"), device="cuda")
        out = torch.full((2 * K * D,), float("nan"), device="cuda")
        assert fv.fv_encode(g, Xd, ref) == fv.FV_OK
        assert fv.fv_encode_noalloc(g, Xd, out) == fv.FV_OK
        torch.cuda.synchronize()
        a, b = ref.cpu().numpy(), out.cpu().numpy()
        assert np.all(np.isfinite(b))
        assert max_err(a, b) <= TOL[fv.FV_PREC_FP32]
    g.close()


def test_noalloc_widened_ranges_match_fv_encode_and_oracle():
    """K=64, D=64, N=100000: the posteriors take 25.6 MB, so the default
    statistics ranges (about 447 slots of 33 KB) do not fit in the fixed
    scratch and the entry point widens them (fewer, longer ranges) until they
    do; the result must still match fv_encode and the FP64 oracle."""
    torch = torch_cuda()
    from gpu_util import oracle_fv
    from paper_1604_03498_gb300 import synth
    K, D, N = 64, 64, 100000
    _, w, mu, var = case(K, D, 10, 42)
    g = fv.fv_gmm_load(w, mu, var, fv.FV_PREC_FP32)
    X = synth.sample_descriptors(w, mu, var, N, seed=600, gmm_frac=0.8)
    Xd = torch.from_numpy(X).cuda()
    ref = torch.full((2 * K * D,), float("nan"), device="cuda")
    out = torch.full((2 * K * D,), float("nan"), device="cuda")
    assert fv.fv_encode(g, Xd, ref) == fv.FV_OK
    assert fv.fv_encode_noalloc(g, Xd, out) == fv.FV_OK
    torch.cuda.synchronize()
    a, b = ref.cpu().numpy(), out.cpu().numpy()
    assert max_err(a, b) <= TOL[fv.FV_PREC_FP32]
    assert max_err(b, oracle_fv(X, w, mu, var)) <= TOL[fv.FV_PREC_FP32]
    g.close()


def test_noalloc_rejects_inputs_beyond_its_fixed_scratch():
    torch = torch_cuda()
    K, D = 512, 64
    _, w, mu, var = case(K, D, 10, 41)
    g = fv.fv_gmm_load(w, mu, var, fv.FV_PREC_FP32)
    X = torch.zeros((20000, D), device="cuda")   # 20000 x 512 x 4 B of posteriors > 32 MiB
    out = torch.zeros(2 * K * D, device="cuda")
    with pytest.raises(fv.FVError) as e:
        fv.fv_encode_noalloc(g, X, out)
    assert e.value.status == fv.FV_ERR_UNSUPPORTED
    assert "32 MiB" in str(e.value)
    g.close()
