"""Write tests/golden/c5_reference.json: FP64 oracle residuals on the held-out warm-start instances.

Instances: n = 50000 points of a 32-component Gaussian mixture in R^64 with Dirichlet(1) weights
(seeds 0..3), X_ij = exp(-||x_i - x_j||^2 / sigma^2), sigma = median pairwise distance over a seeded
sample of 10^6 pairs; k = 32, alpha = max(X), start H0 = Philox Uniform[0,1) (key = instance seed)
* 2 sqrt(mean(X) / k), W0 = H0 (the paper's scaled uniform start).  Recorded: the normalized
residual ||X - W H^T|| / ||X|| of plain regularized HALS every 10 sweeps up to 200, evaluated with
the trace trick (Appendix "Fast Residual Evaluation"; an n x n residual would not fit in memory).
Calls only oracle/ and synth/.  About 8 minutes and 25 GB of memory per instance.

Run:  python tests/golden/make_c5_reference.py [seeds...]
"""

import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import philox  # noqa: E402
from oracle import symnmf as O  # noqa: E402
from synth import gmm_points, kernel_matrix_numpy, median_pair_distance  # noqa: E402

N, D, C, K, SWEEPS, EVERY = 50000, 64, 32, 32, 200, 10


def instance(seed):
    t0 = time.time()
    pts, _ = gmm_points(N, D, C, seed=seed, weights="dirichlet")
    sigma = median_pair_distance(pts, seed=seed)
    X = kernel_matrix_numpy(pts, sigma, block=5000)
    normX2 = float(np.einsum("ij,ij->", X, X))
    alpha = O.default_alpha(X)
    H0 = philox.philox_uniform_factor(N, K, seed) * O.init_scale(X, K)
    out = dict(seed=seed, sigma=sigma, alpha=alpha, normX2=normX2, mean=float(X.mean()), plain_nr={})
    W, H = H0.copy(), H0.copy()
    for t in range(EVERY, SWEEPS + 1, EVERY):
        W, H, _ = O.hals_symnmf(X, H, alpha, EVERY, W0=W, record=False)
        r2 = O.trace_trick_residual_sq(normX2, W.T @ W, H.T @ H, W.T @ (X @ H))
        out["plain_nr"][str(t)] = float(np.sqrt(max(r2, 0.0) / normX2))
        print(seed, t, out["plain_nr"][str(t)], f"{time.time() - t0:.0f}s", flush=True)
    out["seconds"] = time.time() - t0
    return out


def main():
    seeds = [int(a) for a in sys.argv[1:]] or [0, 1, 2, 3]
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c5_reference.json")
    res = dict(n=N, d=D, c=C, k=K, sweeps=SWEEPS, every=EVERY, weights="dirichlet", instances={})
    if os.path.exists(path):
        res = json.load(open(path))
    for s in seeds:
        res["instances"][str(s)] = instance(s)
        with open(path, "w") as f:
            json.dump(res, f, indent=1)


if __name__ == "__main__":
    main()
