"""Write tests/golden/c3_reference.json: FP64 oracle results on the sparse LvS workload.

Instance: stochastic block model, n = 10^6 nodes, 64 equal communities, mean degree 30,
p_in / p_out = 20, unit weights with self-loops, node order shuffled (synth.sbm_csr, seed 0);
k = 64, alpha = max(X) = 1, start H0 = Philox Uniform[0,1) (key 3) * 2 sqrt(mean(X) / k), W0 = H0.
Recorded every 5 outer iterations up to 50:
- plain regularised HALS on the full X (normalized residual by the trace trick);
- LvS-SymNMF with the hybrid sampler, s = ceil(8 k ln k) = 2130 rows, tau = 1/s, Philox key 3.
Calls only oracle/ and synth/.  Takes about 15 minutes on 8 cores.

Run:  python tests/golden/make_c3_reference.py
"""

import json
import math
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import scipy.sparse as sp  # noqa: E402

from oracle import philox  # noqa: E402
from oracle import symnmf as O  # noqa: E402
from synth import lvs_sample_count, sbm_csr  # noqa: E402

N, C, K, ITERS, SEED, EVERY = 1_000_000, 64, 64, 50, 3, 5


def nr_of(Xs, normX2, W, H):
    r2 = O.trace_trick_residual_sq(normX2, W.T @ W, H.T @ H, W.T @ (Xs @ H))
    return math.sqrt(max(r2, 0.0) / normX2)


def main():
    t0 = time.time()
    g = sbm_csr(n=N, c=C, avg_deg=30.0, ratio=20.0, seed=0)
    Xs = sp.csr_matrix((g["val"].astype(np.float64), g["col"], g["row_ptr"]), shape=(N, N))
    normX2 = float(Xs.multiply(Xs).sum())
    mean = float(Xs.sum()) / (float(N) * N)
    alpha = 1.0
    H0 = philox.philox_uniform_factor(N, K, SEED) * (2.0 * math.sqrt(mean / K))
    s = lvs_sample_count(K)
    out = dict(n=N, c=C, k=K, iters=ITERS, seed=SEED, s=s, tau=1.0 / s, nnz=int(Xs.nnz), normX2=normX2,
               mean=mean, alpha=alpha)
    W, H = H0.copy(), H0.copy()
    plain = {}
    for t in range(1, ITERS + 1):
        W, H, _ = O.hals_symnmf(Xs, H, alpha, 1, W0=W, record=False)
        if t % EVERY == 0:
            plain[str(t)] = nr_of(Xs, normX2, W, H)
            print("plain", t, plain[str(t)], time.time() - t0, flush=True)
    out["plain_nr"] = plain
    W, H = H0.copy(), H0.copy()
    lvs = {}
    for t in range(ITERS):
        # one LvS iteration with the draw counters of iteration t
        lev, _ = O.leverage_scores(H)
        smp = O.hybrid_sample(lev, K, s, 1.0 / s, SEED, t, 0)
        Y, G = O.sampled_products(Xs, H, smp["idx"], smp["wt"])
        W = O.hals_update_efficient(W, H, G, Y, alpha)
        lev, _ = O.leverage_scores(W)
        smp = O.hybrid_sample(lev, K, s, 1.0 / s, SEED, t, 1)
        Y, G = O.sampled_products(Xs, W, smp["idx"], smp["wt"])
        H = O.hals_update_efficient(H, W, G, Y, alpha)
        if (t + 1) % EVERY == 0:
            lvs[str(t + 1)] = nr_of(Xs, normX2, W, H)
            print("lvs", t + 1, lvs[str(t + 1)], time.time() - t0, flush=True)
    out["lvs_nr"] = lvs
    out["seconds"] = time.time() - t0
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c3_reference.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
