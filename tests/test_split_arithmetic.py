"""The exactness facts the BF16 form's split products rest on, checked on the
CPU over every bfloat16 value the descriptors can take (|x| < 2^8):

1. x^2 = hi + lo exactly, with hi = bf16(x*x) and lo = bf16(x*x - hi) (for
   |x| >= 2^-59 and x = 0, i.e. while the residual stays a normal number): the
   kernel forms hi with a bf16x2 multiply and lo with a fused multiply-add,
   and feeds both to the tensor cores, so the statistics GEMM sees x^2
   without error (what lets the finalise centre S2 - 2 mu S1 + mu^2 S0
   exactly when a descriptor sits on a mean).
2. For a value q stored as hi + lo (the GMM operand Q = mu/sigma^2 and
   R = -1/(2 sigma^2)), |q - (hi + lo)| <= 2^-16 |q|, so the two products
   per term carry a relative error far below the 2e-3 tolerance.
"""
import numpy as np

from paper_1604_03498_gb300 import synth


def _bf16(v):
    return synth.to_bf16_grid(np.asarray(v, dtype=np.float32)).astype(np.float64)


def _all_bf16_below(limit):
    bits = np.arange(0, 1 << 16, dtype=np.uint32) << 16
    v = bits.view(np.float32)
    v = v[np.isfinite(v)].astype(np.float64)
    a = np.abs(v)
    return v[(a < limit) & ((a >= 2.0 ** -59) | (a == 0))]


def test_square_splits_exactly_into_two_bf16():
    x = _all_bf16_below(256.0)
    sq = x * x                                   # exact in float64 (16 significant bits)
    hi = _bf16(sq)
    lo = _bf16(sq - hi)                          # the FMA's exact residual, rounded to bf16
    assert np.array_equal(hi + lo, sq)


def test_hi_lo_operand_relative_error():
    rng = np.random.default_rng(0)
    q = np.concatenate([rng.normal(0, 1, 200000) / rng.uniform(0.1, 1.0, 200000),
                        -0.5 / rng.uniform(1e-8, 1.0, 200000)])
    hi = _bf16(q)
    lo = _bf16(q - hi)
    rel = np.abs((hi + lo) - q) / np.abs(q)
    assert rel.max() <= 2.0 ** -16
