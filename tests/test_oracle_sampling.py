"""Pins for the oracle's hybrid leverage-score sampler and the sampled products."""

import math

import numpy as np
import scipy.sparse as sp
from scipy import stats

from oracle import symnmf as O
from synth import lvs_sample_count, sbm_csr, uniform_factor


def test_sample_count_formula():
    assert lvs_sample_count(64) == 2130
    assert lvs_sample_count(16) == math.ceil(8 * 16 * math.log(16))


def test_bruteforce_probabilities_reduced_width():
    # enumerate every u of a 12-bit uniform: each row is hit exactly
    # ceil(C_i 2^b / T) - ceil(C_{i-1} 2^b / T) times, i.e. q_i / T up to 2^-b
    lev = np.array([0.01, 0.3, 0.0, 0.12, 0.7, 0.05, 0.22, 0.6])
    k, bits = 2, 12
    words = list(range(1 << bits))
    smp = O.hybrid_sample(lev, k, s=len(words), tau=1.0, seed=0, it=0, side=0, ubits=bits, words=words)
    assert smp["s_D"] == 0
    counts = np.bincount(smp["idx"], minlength=8)
    C = smp["C"].astype(object)
    T = smp["T"]
    prev = 0
    for i in range(8):
        hi = -((-int(C[i]) << bits) // T)
        lo = -((-int(prev) << bits) // T)
        assert counts[i] == hi - lo
        assert abs(counts[i] / 2 ** bits - int(smp["q"][i]) / T) <= 2.0 ** -bits
        prev = C[i]
    assert counts[2] == 0  # zero leverage is never drawn


def test_deterministic_set_threshold_and_order():
    rng = np.random.default_rng(0)
    lev = rng.random(1000) * 0.02
    lev[[5, 900, 17]] = [0.9, 0.5, 0.45]
    k, s = 4, 50
    tau = 0.1  # l_i / k >= 0.1  <=>  l_i >= 0.4
    smp = O.hybrid_sample(lev, k, s, tau, seed=1, it=0, side=0)
    assert list(smp["idx"][: smp["s_D"]]) == [5, 17, 900]
    assert smp["s_D"] == 3 and smp["s_R"] == 47
    np.testing.assert_array_equal(smp["wt"][:3], 1.0)
    assert abs(smp["theta"] - 1.85) < 1e-12
    assert not np.isin(smp["idx"][3:], [5, 17, 900]).any()
    mass = lev.sum() - 1.85
    np.testing.assert_allclose(smp["wt"][3:], mass / (47 * lev[smp["idx"][3:]]), rtol=1e-12)


def test_chi_square_of_philox_draws():
    rng = np.random.default_rng(1)
    lev = rng.random(20)
    smp = O.hybrid_sample(lev, k=100, s=200000, tau=1.0, seed=3, it=2, side=1)
    counts = np.bincount(smp["idx"], minlength=20)
    p = smp["q"].astype(np.float64) / smp["T"]
    chi = stats.chisquare(counts, p * counts.sum())
    assert chi.pvalue > 1e-4


def test_unbiased_sampled_gram():
    # E[F^T S^T S F] = F^T F (hybrid sampling keeps the estimator unbiased)
    rng = np.random.default_rng(2)
    F = rng.random((300, 3))
    F[:4] *= 8.0
    lev, _ = O.leverage_scores(F)
    G = F.T @ F
    acc = np.zeros((3, 3))
    reps = 3000
    for it in range(reps):
        smp = O.hybrid_sample(lev, 3, 40, 1.0 / 40, seed=11, it=it, side=0)
        Fs = F[smp["idx"]]
        acc += Fs.T @ (smp["wt"][:, None] * Fs)
    mean = acc / reps
    assert np.abs(mean - G).max() / np.abs(G).max() < 0.03


def test_sampled_normal_equations_match_stacked_problem():
    # || [S H; sqrt(a) I] W^T - [S X; sqrt(a) H^T] ||^2 has normal equations
    # (H^T S^T S H + a I) W^T = H^T S^T S X + a H^T  (Section LvS, regularised sampling)
    rng = np.random.default_rng(3)
    n, k, a = 60, 4, 0.6
    A = rng.random((n, n))
    X = 0.5 * (A + A.T)
    H = rng.random((n, k))
    lev, _ = O.leverage_scores(H)
    smp = O.hybrid_sample(lev, k, 25, 0.05, seed=4, it=0, side=0)
    S = np.zeros((smp["idx"].shape[0], n))
    S[np.arange(S.shape[0]), smp["idx"]] = np.sqrt(smp["wt"])
    Acoef = np.vstack([S @ H, math.sqrt(a) * np.eye(k)])
    B = np.vstack([S @ X, math.sqrt(a) * H.T])
    Gn = Acoef.T @ Acoef
    Yn = (Acoef.T @ B).T
    Y, G = O.sampled_products(X, H, smp["idx"], smp["wt"])
    np.testing.assert_allclose(G + a * np.eye(k), Gn, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(Y + a * H, Yn, rtol=1e-12, atol=1e-12)


def test_sparse_and_dense_sampled_products_agree():
    g = sbm_csr(n=2000, c=8, avg_deg=10, ratio=10, seed=0)
    Xs = sp.csr_matrix((g["val"].astype(np.float64), g["col"], g["row_ptr"]), shape=(2000, 2000))
    assert abs(Xs - Xs.T).max() == 0
    H = uniform_factor(2000, 5, seed=0)
    lev, _ = O.leverage_scores(H)
    smp = O.hybrid_sample(lev, 5, 80, 1.0 / 80, seed=0, it=0, side=0)
    Y1, G1 = O.sampled_products(Xs, H, smp["idx"], smp["wt"])
    Y2, G2 = O.sampled_products(Xs.toarray(), H, smp["idx"], smp["wt"])
    np.testing.assert_allclose(Y1, Y2, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(G1, G2, rtol=1e-12)


def test_sbm_generator_shape():
    g = sbm_csr(n=6400, c=64, avg_deg=30, ratio=20, seed=1)
    deg = np.diff(g["row_ptr"])
    assert abs(deg.mean() - 31.0) < 1.0  # 30 expected neighbours + the self loop
    lab = g["labels"]
    rows = np.repeat(np.arange(6400), deg)
    intra = (lab[rows] == lab[g["col"]]).mean()
    # expected share of intra-community entries: ((n_c - 1) p_in + 1) / 31 = (7.2 + 1) / 31
    assert 0.15 < intra < 0.5


def test_lvs_symnmf_closes_most_of_the_gap_to_full_hals_on_sbm():
    g = sbm_csr(n=3000, c=6, avg_deg=40, ratio=30, seed=2)
    X = sp.csr_matrix((g["val"].astype(np.float64), g["col"], g["row_ptr"]), shape=(3000, 3000))
    Xd = X.toarray()
    H0 = uniform_factor(3000, 6, seed=2) * O.init_scale(Xd, 6)
    alpha = 1.0
    nr0 = O.normalized_residual(Xd, H0, H0)
    Wf, Hf, _ = O.hals_symnmf(Xd, H0, alpha, 20, record=False)
    nr_full = O.normalized_residual(Xd, Wf, Hf)
    W, H = O.lvs_symnmf(X, H0, alpha, iters=20, s=1000, tau=1.0 / 1000, seed=5)
    assert O.normalized_residual(Xd, W, H) <= nr_full + 0.5 * (nr0 - nr_full)
