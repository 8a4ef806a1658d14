"""Write the small golden fixtures of tests/golden/ from the FP64 oracle.

The paper prints no worked example or Fisher-vector values (Sec. 3.1 gives
Algorithm 1 only), so every stored expectation here is the oracle's output on
a seeded synthetic input; the oracle itself is pinned by the oracle tests.
Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import oracle  # noqa: E402
from paper_1604_03498_gb300 import synth  # noqa: E402

CASES = [
    # name, N, D, K, seed, gmm_frac
    ("tiny_n5_d3_k2", 5, 3, 2, 1, 1.0),
    ("ragged_n130_d16_k8", 130, 16, 8, 2, 0.8),
    ("single_n1_d64_k64", 1, 64, 64, 3, 1.0),
]


def main():
    here = os.path.dirname(os.path.abspath(__file__))
    for name, N, D, K, seed, frac in CASES:
        w, mu, var = synth.make_gmm(K, D, seed=seed)
        X = synth.sample_descriptors(w, mu, var, N, seed=seed, gmm_frac=frac)
        r = oracle.encode(X, w, mu, var)
        doc = {
            "source": "oracle/fv_oracle.c (Algorithm 1, Sec. 3.1; normalisation of Sec. 4)",
            "N": N, "D": D, "K": K,
            "X": X.astype(np.float64).ravel().tolist(),
            "w": w.astype(np.float64).tolist(),
            "mu": mu.astype(np.float64).ravel().tolist(),
            "var": var.astype(np.float64).ravel().tolist(),
            "fv": r["fv"].tolist(),
        }
        with open(os.path.join(here, name + ".json"), "w") as f:
            json.dump(doc, f)
        print("wrote", name)


if __name__ == "__main__":
    main()
