"""The fused BF16 encoder's barrier protocol, run on the CPU model in
encoder_protocol_model.py: randomised interleavings of every role for 1-4
CTA clusters, one and two Y stages and units of 1 to 700 rows must finish
with no buffer overwritten in use, no stale read, no deadlock and every
unit's statistics written out, for the plain BF16 and the BF16X2 (hi + lo
posteriors in two 64-row halves) protocols; and the model must catch a
protocol with one of the kernel's waits taken out (so a passing run means
something).
The waits on LEMPTY and TEMPTY are not in the second list: the tile chain
already implies them (a stage is rebuilt only after the statistics GEMM
that follows the softmax's release, and a new unit's first statistics MMA
waits for gamma^T, written after the flush), so the kernel keeps them for
robustness only."""
import random

import pytest

import encoder_protocol_model as model


def _cases(seed, n):
    rng = random.Random(seed)
    for t in range(n):
        S = rng.choice([1, 2, 3, 4])
        nstage = rng.choice([1, 2])
        units = [rng.choice([1, 100, 128, 129, 256, 300, 700]) for _ in range(rng.randint(1, 5))]
        yield units, S, nstage, t, rng.random() < 0.5


def test_protocol_holds_under_random_interleavings():
    for units, S, nstage, t, glo in _cases(1, 200):
        model.run(units, S, nstage, t, glo=glo)


@pytest.mark.parametrize("drop,glo", [("builder_stfree", False), ("l_xrfree", False), ("softmax_gfree", False),
                                      ("softmax_hxfree", False), ("softmax_gfree", True), ("softmax_tempty", True)])
def test_model_catches_a_missing_wait(drop, glo):
    for units, S, nstage, t, _ in _cases(7, 300):
        try:
            model.run(units, S, nstage, t, drop=frozenset([drop]), glo=glo)
        except (model.Fail, AssertionError):
            return
    pytest.fail(f"no interleaving exposed the protocol without the {drop} wait")
