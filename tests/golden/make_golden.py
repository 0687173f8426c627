"""Writes the stored expected values under tests/golden/ from the FP64 oracle
only (no CUDA code): a small seeded Ising problem (App. A's pseudo-likelihood
with the Laplace prior) with every pair's exact gain and maximiser at the
W = 0 start, the start objective, the exhaustive best pairs (Algorithm 3's
base case) and the objective after one sequential update sweep over them
(Algorithm 2).  Run from the repository root:

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle  # noqa: E402
from paper_2401_01404_gb300 import inputs  # noqa: E402

N, M, SEED, C = 12, 64, 404, 0.5


def main():
    edges = inputs.erdos_renyi(N, 3, inputs.rng(SEED, inputs.GRAPH))
    w = inputs.rng(SEED, inputs.COUPLINGS).normal(0, 0.5, len(edges))
    h = inputs.rng(SEED, inputs.FIELDS).normal(0, 0.1, N)
    X = inputs.gibbs_ising(N, edges, w, h, M, 200, SEED)
    lam = inputs.default_lambda(N, M, C)
    o = oracle.IsingOracle(X, lam, w_clamp=5.0)
    h0 = o.h.copy()
    pairs = oracle.all_pairs(np.arange(N))
    g, ws = o.score(pairs)
    obj0 = o.objective()
    D = o.dist_matrix()
    best = oracle.exhaustive_best(D, N)
    o.update(best)
    out = {
        "source": "tests/golden/make_golden.py (FP64 oracle: App. A pseudo-likelihood, Laplace prior; "
                  "Algorithm 3's exhaustive base case; one sequential sweep of Algorithm 2)",
        "N": N, "M": M, "lambda": lam, "w_clamp": 5.0,
        "X": X.astype(int).tolist(),
        "fields_w0": h0.tolist(),
        "pairs": pairs.tolist(), "gain": g.tolist(), "w": ws.tolist(),
        "objective_w0": obj0,
        "best_pairs": np.asarray(best).tolist(),
        "objective_after_sweep": o.objective(),
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "ising_n12_m64.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=None, separators=(",", ":"))
        f.write("\n")
    print(path)


if __name__ == "__main__":
    main()
