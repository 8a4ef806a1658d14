"""CPU-side checks of the C ABI: the library builds, loads and exports every
function include/fv.h declares; argument validation answers without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1604_03498_gb300 import fv

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            names |= set(re.findall(r"FV_API\s+[\w\s\*]*?\b(fv_\w+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("fv_gmm_load", "fv_gmm_free", "fv_encode", "fv_encode_batch", "fv_last_error"):
        assert n in names


@pytest.mark.parametrize("name", _declared())
def test_library_exports_every_declared_symbol(name):
    L = fv.lib()
    assert hasattr(L, name), f"{name} declared in include/ but not exported"


def test_limits_without_gpu():
    assert fv.fv_limits(fv.FV_PREC_FP32)[0] >= 512
    K, D = fv.fv_limits(fv.FV_PREC_BF16)
    assert K >= 512 and D >= 80
    with pytest.raises(fv.FVError) as e:
        fv.fv_limits(7)
    assert e.value.status == fv.FV_ERR_INVALID


@pytest.mark.parametrize("case", ["bad_weights", "bad_sum", "bad_var", "nan_mean", "too_big"])
def test_gmm_validation_rejects_before_any_device_work(case):
    K, D = 4, 3
    w = np.full(K, 0.25, np.float32)
    mu = np.zeros((K, D), np.float32)
    var = np.ones((K, D), np.float32)
    prec = fv.FV_PREC_FP32
    if case == "bad_weights":
        w[0] = -0.1
    elif case == "bad_sum":
        w[:] = 0.3
    elif case == "bad_var":
        var[1, 2] = 0.0
    elif case == "nan_mean":
        mu[2, 0] = np.nan
    else:
        K, D = 4, 200
        w = np.full(K, 0.25, np.float32)
        mu = np.zeros((K, D), np.float32)
        var = np.ones((K, D), np.float32)
        prec = fv.FV_PREC_BF16
    with pytest.raises(fv.FVError) as e:
        fv.fv_gmm_load(w, mu, var, prec)
    want = fv.FV_ERR_UNSUPPORTED if case == "too_big" else fv.FV_ERR_INVALID
    assert e.value.status == want
    assert fv.fv_last_error()


def test_null_handle_is_rejected():
    L = fv.lib()
    out = np.zeros(8, np.float32)
    st = L.fv_encode(None, None, 0, 0, out.ctypes.data, 0, None)
    assert st == fv.FV_ERR_INVALID
