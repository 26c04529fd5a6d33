"""Write tests/golden/c2_reference.json: FP64 oracle results on the LAI benchmark instance.

Instance: n = 20000 points of a 20-component Gaussian mixture in R^50 (seed 0),
X_ij = exp(-||x_i - x_j||^2 / sigma^2), sigma = median pairwise distance over a
seeded sample of 10^6 pairs; k = 20, l = 2k + 10 = 50, q = 2, 200 sweeps,
alpha = max(X) = 1, start H0 = Philox Uniform[0,1) (key 1) * 2 sqrt(mean(X) / k),
W0 = H0.  Calls only oracle/ and synth/.

Run:  python tests/golden/make_c2_reference.py
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

N, D, C, K, L, Q, SWEEPS, SEED = 20000, 50, 20, 20, 50, 2, 200, 1


def main():
    t0 = time.time()
    pts, _ = gmm_points(N, D, C, seed=0)
    sigma = median_pair_distance(pts, seed=0)
    X = kernel_matrix_numpy(pts, sigma)
    alpha = O.default_alpha(X)
    H0 = philox.philox_uniform_factor(N, K, SEED) * O.init_scale(X, K)
    out = dict(n=N, d=D, c=C, k=K, l=L, q=Q, sweeps=SWEEPS, seed=SEED, sigma=sigma, alpha=alpha,
               normX2=float((X * X).sum()), mean=float(X.mean()))
    W, H, objs = O.hals_symnmf(X, H0, alpha, SWEEPS)
    out["plain_nr"] = O.normalized_residual(X, W, H)
    out["plain_obj"] = {str(t): objs[t - 1] for t in (1, 10, 50, 100, 200)}
    Om = philox.philox_gaussian(N, L, SEED)
    U, lam = O.apx_evd(X, Om, Q)
    W2, H2, objs2 = O.lai_symnmf(U, lam, H0, alpha, SWEEPS)
    out["lai_nr_true"] = O.normalized_residual(X, W2, H2)
    out["lai_obj"] = {str(t): objs2[t - 1] for t in (1, 10, 50, 100, 200)}
    out["lai_normX2"] = float((lam ** 2).sum())
    out["seconds"] = time.time() - t0
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c2_reference.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
