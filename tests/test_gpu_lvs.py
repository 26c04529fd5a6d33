"""GPU parity of LvS-SymNMF: leverage scores, the hybrid sampler (bit-exact) and sampled updates."""

import numpy as np
import pytest
import scipy.sparse as sp
import torch

from oracle import symnmf as O
from synth import lvs_sample_count, sbm_csr, uniform_factor

from ._gpu_util import np64, rel_err, t32

pytestmark = pytest.mark.gpu


def _sbm(n, c, k, seed, deg=30.0):
    g = sbm_csr(n=n, c=c, avg_deg=deg, ratio=20, seed=seed)
    Xs = sp.csr_matrix((g["val"].astype(np.float64), g["col"], g["row_ptr"]), shape=(n, n))
    dev = dict(row_ptr=torch.tensor(g["row_ptr"], device="cuda"), col=torch.tensor(g["col"], device="cuda"),
               val=torch.tensor(g["val"], device="cuda"))
    return g, Xs, dev


def _solver(S, dev, n, k, **kw):
    return S.Solver(csr=(dev["row_ptr"], dev["col"], dev["val"]), k=k, n=n, **kw)


@pytest.mark.parametrize("n,k", [(20000, 16), (1031, 64), (777, 50), (300, 5), (3, 2)])
def test_leverage_scores(S, n, k):
    # ragged n against the 256-row tiles of the row pass, 16-byte rows (k % 4 == 0) and not
    _, Xs, dev = _sbm(n, 16 if n >= 1000 else 1, k, seed=0, deg=min(30.0, n / 8))
    s = _solver(S, dev, n, k, seed=3)
    Hi = uniform_factor(n, k, seed=1)
    s.set_factors(t32(Hi))
    lev = np64(s.leverage(0))
    ref, _ = O.leverage_scores(Hi.astype(np.float32).astype(np.float64))
    np.testing.assert_allclose(lev, ref, rtol=2e-4, atol=1e-9)
    assert abs(lev.sum() - k) < 1e-3


@pytest.mark.parametrize("n,k,tau_mode", [(20000, 16, "1/s"), (20000, 16, "1"), (1000, 4, "big"),
                                          (333, 5, "1/s")])
def test_sampler_bit_exact_with_oracle_scores(S, n, k, tau_mode):
    g, Xs, dev = _sbm(max(n, 64), 8, k, seed=1, deg=10.0)
    n = g["n"]
    rng = np.random.default_rng(n + k)
    F = rng.random((n, k))
    F[:7] *= 30.0  # a few heavy rows for the deterministic part
    lev, _ = O.leverage_scores(F)
    s_cnt = lvs_sample_count(k)
    tau = {"1/s": 1.0 / s_cnt, "1": 1.0, "big": 0.0}[tau_mode]
    s = _solver(S, dev, n, k, seed=2024)
    for it, side in [(0, 0), (3, 1), (17, 0)]:
        got = s.lvs_sample(side, it, tau, s_cnt, lev_in=lev)
        ref = O.hybrid_sample(lev, k, s_cnt, tau, seed=2024, it=it, side=side)
        assert got["s_D"] == ref["s_D"]
        assert got["s_tot"] == ref["idx"].shape[0]
        np.testing.assert_array_equal(got["idx"], ref["idx"])
        np.testing.assert_allclose(got["wt"], ref["wt"], rtol=1e-6)
        assert got["theta"] == pytest.approx(ref["theta"], rel=1e-12, abs=1e-300)


def test_sampler_edge_cases(S):
    g, Xs, dev = _sbm(500, 4, 3, seed=2, deg=8.0)
    n = g["n"]
    s = _solver(S, dev, n, 3, seed=7)
    lev = np.zeros(n)
    lev[[3, 10, 11]] = [1.0, 1.0, 1.0]
    # all mass deterministic: no draws
    got = s.lvs_sample(0, 0, 0.1, 50, lev_in=lev)
    ref = O.hybrid_sample(lev, 3, 50, 0.1, seed=7, it=0, side=0)
    assert got["s_D"] == 3 and got["s_tot"] == 3
    np.testing.assert_array_equal(got["idx"], ref["idx"])
    # s = 0
    got = s.lvs_sample(0, 0, 1.0, 0, lev_in=np.full(n, 3.0 / n))
    assert got["s_tot"] == 0


def test_sampled_update_matches_oracle(S):
    n, k = 20000, 16
    _, Xs, dev = _sbm(n, 16, k, seed=3)
    s = _solver(S, dev, n, k, seed=11, use_graph=False)
    Hi = uniform_factor(n, k, seed=4) * 0.1
    s.set_factors(t32(Hi))
    H0 = Hi.astype(np.float32).astype(np.float64)
    lev, _ = O.leverage_scores(H0)
    s_cnt = lvs_sample_count(k)
    got = s.lvs_sample(0, 0, 1.0 / s_cnt, s_cnt, lev_in=lev)
    s.lvs_update(0)
    Hg, Wg = (np64(t) for t in s.factors())
    idx, wt = got["idx"].astype(np.int64), got["wt"].astype(np.float64)
    Y, G = O.sampled_products(Xs, H0, idx, wt)
    alpha = 1.0
    Wref = O.hals_update_efficient(H0, H0, G, Y, alpha)
    np.testing.assert_allclose(Wg, Wref, rtol=1e-4, atol=1e-6)


def test_lvs_iterations_reduce_residual_like_oracle(S):
    n, k = 20000, 16
    g, Xs, dev = _sbm(n, 16, k, seed=5)
    s_cnt = lvs_sample_count(k)
    Hi = uniform_factor(n, k, seed=6) * 0.05
    s = _solver(S, dev, n, k, seed=13)
    s.set_factors(t32(Hi))
    s.lvs_iterate(10, 1.0 / s_cnt, s_cnt)
    nr_gpu, _ = s.residual(S.SRC_X)
    W, H = O.lvs_symnmf(Xs, Hi.astype(np.float32).astype(np.float64), 1.0, 10, s_cnt, 1.0 / s_cnt, seed=13)
    Xd = None
    # residual of the oracle run via the trace trick on the sparse X
    XH = Xs @ H
    r2 = Xs.multiply(Xs).sum() + np.trace((W.T @ W) @ (H.T @ H)) - 2 * np.trace(W.T @ XH)
    nr_oracle = np.sqrt(max(r2, 0) / Xs.multiply(Xs).sum())
    assert abs(nr_gpu - nr_oracle) < 5e-3
    del Xd
