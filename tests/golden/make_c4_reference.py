"""Write tests/golden/c4_reference.json: FP64 oracle results on the batched workload.

Instance: 64 dense SBM problems (synth.batched_problem_specs(64, seed 0): n log-uniform in
[500, 8000], k from {8, 12, 16, 24, 32}); problem p is synth.dense_sbm(n_p, k_p, seed 1000 + p)
(k_p equal communities, p_in = 0.3, p_out = 0.015, unit diagonal), alpha = max(X) = 1.
Each problem has 4 restarts; restart r starts from Philox Uniform[0,1) with key p + r, scaled
by 2 sqrt(mean(X) / k), W0 = H0.  Recorded: the normalized residual ||X - W H^T|| / ||X|| of
every (problem, restart) after 100 regularised HALS sweeps, problem-major.
Calls only oracle/ and synth/.  A few minutes on 8 cores.

Run:  python tests/golden/make_c4_reference.py
"""

import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import philox  # noqa: E402
from oracle import symnmf as O  # noqa: E402
from synth import batched_problem_specs, dense_sbm  # noqa: E402

SWEEPS, RESTARTS = 100, 4


def main():
    t0 = time.time()
    specs = batched_problem_specs(64, seed=0)
    nr = []
    for p, sp in enumerate(specs):
        n, k = sp["n"], sp["k"]
        A, _ = dense_sbm(n, k, seed=1000 + p)
        X = A.astype("float64")
        alpha = O.default_alpha(X)
        for r in range(RESTARTS):
            H0 = philox.philox_uniform_factor(n, k, p + r) * O.init_scale(X, k)
            W, H, _ = O.hals_symnmf(X, H0, alpha, SWEEPS, record=False)
            nr.append(O.normalized_residual(X, W, H))
        print(p, n, k, nr[-4:], time.time() - t0, flush=True)
    out = dict(nprob=64, restarts=RESTARTS, sweeps=SWEEPS, ns=[s["n"] for s in specs], ks=[s["k"] for s in specs],
               nr=nr, seconds=time.time() - t0)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "c4_reference.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
