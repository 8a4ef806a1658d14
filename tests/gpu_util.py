"""Shared helpers of the GPU tests (no method arithmetic here)."""
import numpy as np

import oracle
from paper_1604_03498_gb300 import fv, synth

TOL = {fv.FV_PREC_FP32: 1e-4, fv.FV_PREC_BF16: 2e-3, fv.FV_PREC_BF16X2: 2e-3}


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU test run without a CUDA device"
    return torch


def case(K, D, N, seed=0, frac=0.8):
    w, mu, var = synth.make_gmm(K, D, seed=seed)
    X = synth.sample_descriptors(w, mu, var, N, seed=seed, gmm_frac=frac)
    return X, w, mu, var


def gpu_encode(prec, X, w, mu, var, on_device=True):
    torch = torch_cuda()
    g = fv.fv_gmm_load(w, mu, var, prec)
    K, D = mu.shape
    if on_device:
        Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()
        out = torch.full((2 * K * D,), float("nan"), device="cuda")
        st = fv.fv_encode(g, Xd, out)
        torch.cuda.synchronize()
        res = out.cpu().numpy()
    else:
        res = np.full(2 * K * D, np.nan, np.float32)
        st = fv.fv_encode(g, np.ascontiguousarray(X, dtype=np.float32), res)
    g.close()
    return st, res


def gpu_encode_batch(prec, frames, w, mu, var):
    torch = torch_cuda()
    g = fv.fv_gmm_load(w, mu, var, prec)
    K, D = mu.shape
    offs = np.zeros(len(frames) + 1, np.int64)
    offs[1:] = np.cumsum([f.shape[0] for f in frames])
    Xp = np.concatenate([f.reshape(-1, D) for f in frames], 0).astype(np.float32) if offs[-1] else np.zeros((1, D), np.float32)
    Xd = torch.from_numpy(np.ascontiguousarray(Xp)).cuda()
    out = torch.full((len(frames), 2 * K * D), float("nan"), device="cuda")
    st = fv.fv_encode_batch(g, Xd, offs, out)
    torch.cuda.synchronize()
    g.close()
    return st, out.cpu().numpy()


def oracle_fv(X, w, mu, var):
    return oracle.encode(X, w, mu, var)["fv"]


def max_err(a, b):
    return float(np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64)).max())
