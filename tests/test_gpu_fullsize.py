"""Parity at the full size of the sparse LvS workload: n = 10^6 SBM nodes, k = 64.

The CSR graph is the stochastic block model of the LvS experiments (64 communities, mean degree 30,
p_in / p_out = 20, unit weights, self-loops).  From one seeded start the GPU runs
- one full-X sweep (CSR product, HALS and Grams, both halves), and
- one LvS W-half fed the oracle's leverage scores;
the FP64 oracle runs the same steps on the same inputs.  Compared:
- the sweep's surrogate objective (1e-4 relative), W and H on 4096 sampled rows;
- the GPU's leverage scores;
- the sampled indices (bit-exact);
- the LvS-updated W on 65536 sampled rows (rows are independent once Y and G are fixed).
"""

import numpy as np
import pytest
import scipy.sparse as sp
import torch

from oracle import symnmf as O
from synth import lvs_sample_count, sbm_csr, uniform_factor

from ._gpu_util import np64, t32

pytestmark = pytest.mark.gpu

N_FULL, K_FULL = 1_000_000, 64


@pytest.fixture(scope="module")
def sbm_full():
    g = sbm_csr(n=N_FULL, c=64, avg_deg=30.0, ratio=20.0, seed=0)
    Xs = sp.csr_matrix((g["val"].astype(np.float64), g["col"], g["row_ptr"]), shape=(N_FULL, N_FULL))
    dev = dict(row_ptr=torch.tensor(g["row_ptr"], device="cuda"), col=torch.tensor(g["col"], device="cuda"),
               val=torch.tensor(g["val"], device="cuda"))
    return Xs, dev


def _start(Xs, seed):
    Hi = uniform_factor(N_FULL, K_FULL, seed=seed, scale=O.init_scale(Xs, K_FULL))
    return Hi.astype(np.float32).astype(np.float64)  # the GPU holds FP32 factors


def _solver(S, dev, seed):
    return S.Solver(csr=(dev["row_ptr"], dev["col"], dev["val"]), k=K_FULL, n=N_FULL, seed=seed,
                    use_graph=False)


def test_full_sweep_at_full_size(S, sbm_full):
    Xs, dev = sbm_full
    H0 = _start(Xs, seed=31)
    s = _solver(S, dev, seed=5)
    s.set_factors(t32(H0))
    obj = s.sweep(1, S.SRC_X, record=True)
    Hg, Wg = (np64(t) for t in s.factors())
    alpha = 1.0  # max(X) of unit weights
    W1 = O.hals_update_efficient(H0, H0, H0.T @ H0, Xs @ H0, alpha)
    H1 = O.hals_update_efficient(H0, W1, W1.T @ W1, Xs @ W1, alpha)
    normX2 = float(Xs.multiply(Xs).sum())
    ref = O.trace_trick_residual_sq(normX2, W1.T @ W1, H1.T @ H1, W1.T @ (Xs @ H1))
    ref += alpha * float(((W1 - H1) ** 2).sum())
    assert abs(obj[0] - ref) <= 1e-4 * abs(ref), (obj[0], ref)
    rows = np.random.default_rng(1).choice(N_FULL, size=4096, replace=False)
    for got, want in ((Wg, W1), (Hg, H1)):
        np.testing.assert_allclose(got[rows], want[rows], rtol=1e-3, atol=1e-5 * np.abs(want).max())


def test_lvs_half_at_full_size(S, sbm_full):
    Xs, dev = sbm_full
    H0 = _start(Xs, seed=32)
    s = _solver(S, dev, seed=2024)
    s.set_factors(t32(H0))
    lev_ref, full_rank = O.leverage_scores(H0)
    assert full_rank
    np.testing.assert_allclose(np64(s.leverage(0)), lev_ref, rtol=2e-4, atol=1e-12)
    s_cnt = lvs_sample_count(K_FULL)
    tau = 1.0 / s_cnt
    got = s.lvs_sample(0, 0, tau, s_cnt, lev_in=lev_ref)
    smp = O.hybrid_sample(lev_ref, K_FULL, s_cnt, tau, seed=2024, it=0, side=0)
    assert got["s_D"] == smp["s_D"] and got["s_tot"] == smp["idx"].shape[0]
    np.testing.assert_array_equal(got["idx"], smp["idx"])
    np.testing.assert_allclose(got["wt"], smp["wt"], rtol=1e-6)
    s.lvs_update(0)
    _, Wg = (np64(t) for t in s.factors())
    Y, G = O.sampled_products(Xs, H0, smp["idx"], smp["wt"])
    # with Y and G fixed the update is row by row: the oracle runs it on a sample of rows
    rows = np.sort(np.random.default_rng(2).choice(N_FULL, size=65536, replace=False))
    Wref = O.hals_update_efficient(H0[rows], H0[rows], G, Y[rows], 1.0)
    np.testing.assert_allclose(Wg[rows], Wref, rtol=1e-3, atol=1e-5 * np.abs(Wref).max())
