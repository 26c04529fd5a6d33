"""Pins for the oracle's range finder, Apx-EVD, LAI products and leverage scores."""

import numpy as np
import pytest

from oracle import symnmf as O
from synth import gaussian_sketch, gmm_points, kernel_matrix_numpy, median_pair_distance, planted_dense, uniform_factor


def _gmm(n, seed):
    pts, labels = gmm_points(n, 8, 5, seed=seed)
    return kernel_matrix_numpy(pts, median_pair_distance(pts, seed=seed)), labels


def _lowrank_sym(n, r, seed):
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((n, r))
    d = rng.uniform(0.5, 2.0, size=r) * rng.choice([-1, 1], size=r)
    return (B * d) @ B.T


def test_exact_range_capture_when_rank_at_most_l():
    X = _lowrank_sym(300, 12, seed=0)
    U, lam = O.apx_evd(X, gaussian_sketch(300, 20, seed=1), q=2)
    err = np.linalg.norm(X - U @ np.diag(lam) @ U.T) / np.linalg.norm(X)
    assert err <= 1e-10
    np.testing.assert_allclose(U.T @ U, np.eye(20), atol=1e-10)


def test_planted_rank_k_captured():
    X, H0, _ = planted_dense(n=400, k=8, sigma=0.0, seed=2)
    U, lam = O.apx_evd(X, gaussian_sketch(400, 26, seed=3), q=1)
    assert np.linalg.norm(X - U @ np.diag(lam) @ U.T) / np.linalg.norm(X) <= 1e-10


def test_lai_product_is_projected_operator():
    # U Lambda U^T = P X P with P = Q Q^T (Alg. Apx-EVD)
    pts, _ = gmm_points(300, 5, 4, seed=0)
    X = kernel_matrix_numpy(pts, median_pair_distance(pts, seed=0))
    Om = gaussian_sketch(300, 15, seed=4)
    Q = O.rrf(X, Om, q=2)
    U, lam = O.apx_evd(X, Om, q=2)
    P = Q @ Q.T
    F = np.random.default_rng(0).random((300, 6))
    np.testing.assert_allclose(O.lai_product(U, lam, F), P @ X @ P @ F, rtol=1e-9, atol=1e-10)


def test_qb_residual_identity():
    # ||Q B - X||^2 = ||X||^2 - ||B||^2 for B = Q^T X (Ada-RRF appendix)
    X = _lowrank_sym(200, 30, seed=5) + 0.01 * np.eye(200)
    Q = O.rrf(X, gaussian_sketch(200, 12, seed=6), q=1)
    B = Q.T @ X
    lhs = np.linalg.norm(Q @ B - X) ** 2
    rhs = np.linalg.norm(X) ** 2 - np.linalg.norm(B) ** 2
    assert abs(lhs - rhs) <= 1e-9 * np.linalg.norm(X) ** 2


def test_evd_projection_bound():
    # ||X - P X P|| <= 2 ||X - P X|| (Section 'Approximation Errors for LAI-NMF')
    pts, _ = gmm_points(250, 6, 5, seed=3)
    X = kernel_matrix_numpy(pts, median_pair_distance(pts, seed=3))
    Q = O.rrf(X, gaussian_sketch(250, 10, seed=7), q=0)
    P = Q @ Q.T
    assert np.linalg.norm(X - P @ X @ P) <= 2 * np.linalg.norm(X - P @ X) + 1e-12


def test_lai_iterates_equal_full_iterates_when_range_captured():
    X, _, _ = planted_dense(n=300, k=6, sigma=0.0, seed=4)
    alpha = O.default_alpha(X)
    U, lam = O.apx_evd(X, gaussian_sketch(300, 16, seed=8), q=2)
    H0 = uniform_factor(300, 6, seed=9) * O.init_scale(X, 6)
    W1, H1, o1 = O.hals_symnmf(X, H0, alpha, 100)
    W2, H2, o2 = O.lai_symnmf(U, lam, H0, alpha, 100)
    np.testing.assert_allclose(H2, H1, rtol=1e-8, atol=1e-9)
    np.testing.assert_allclose(o2, o1, rtol=1e-8)


def test_leverage_scores_match_householder_and_svd():
    rng = np.random.default_rng(10)
    F = rng.random((500, 9))
    lev, full = O.leverage_scores(F)
    assert full
    Qh, _ = np.linalg.qr(F)
    np.testing.assert_allclose(lev, (Qh ** 2).sum(1), rtol=1e-10, atol=1e-14)
    Us, _, _ = np.linalg.svd(F, full_matrices=False)
    np.testing.assert_allclose(lev, (Us ** 2).sum(1), rtol=1e-10, atol=1e-14)
    assert abs(lev.sum() - 9) < 1e-10
    assert lev.min() >= 0 and lev.max() <= 1 + 1e-12


def test_leverage_scores_rank_deficient():
    rng = np.random.default_rng(11)
    F = rng.random((200, 6))
    F[:, 3] = 0.0
    lev, full = O.leverage_scores(F)
    assert not full
    assert abs(lev.sum() - 5) < 1e-9
    Us, s, _ = np.linalg.svd(F, full_matrices=False)
    r = (s > 1e-10 * s[0]).sum()
    np.testing.assert_allclose(lev, (Us[:, :r] ** 2).sum(1), rtol=1e-9, atol=1e-13)


def _projector_distance(Q1, Q2):
    return float(np.linalg.norm(Q1 @ Q1.T - Q2 @ Q2.T, 2))


def test_ada_rrf_without_stopping_is_the_fixed_q_range_finder():
    # never stopping (tol = -inf) after q_max checks leaves the basis of Alg. RRF with q = q_max
    rng = np.random.default_rng(21)
    n, l = 300, 12
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    X = (V * np.exp(-np.arange(n) / 15.0)) @ V.T
    Om = rng.standard_normal((n, l))
    for q in (0, 1, 3):
        Qa, hist, passes = O.ada_rrf(X, Om, q, tol=-np.inf)
        assert len(hist) == q and passes == 1 + 2 * q
        assert _projector_distance(Qa, O.rrf(X, Om, q)) < 1e-10


def test_ada_rrf_residuals_are_the_qb_residuals_of_the_checked_bases():
    # each recorded residual is ||X - Q Q^T X|| / ||X|| of the basis checked, computed directly
    rng = np.random.default_rng(22)
    n, l = 200, 10
    A = rng.standard_normal((n, 30))
    X = A @ A.T + 0.01 * np.eye(n)
    Om = rng.standard_normal((n, l))
    _, hist, _ = O.ada_rrf(X, Om, 4, tol=-np.inf)
    Q, _ = np.linalg.qr(X @ Om)
    for j in range(4):
        direct = np.linalg.norm(X - Q @ (Q.T @ X)) / np.linalg.norm(X)
        assert hist[j] == pytest.approx(direct, rel=1e-8, abs=1e-12)
        Q, _ = np.linalg.qr(X @ Q)
        Q, _ = np.linalg.qr(X @ Q)


def test_ada_rrf_stops_once_the_residual_stalls():
    # rank(X) <= l: the first check already captures X (residual ~ 0), the second finds no
    # further decrease and stops; the EVD then reproduces X exactly
    X, _, _ = planted_dense(n=300, k=6, sigma=0.0, seed=4)
    Om = np.random.default_rng(23).standard_normal((300, 12))
    Q, hist, passes = O.ada_rrf(X, Om, 10, tol=1e-3)
    assert len(hist) == 2 and hist[0] < 1e-12 and passes == 4
    U, lam, _, passes_evd = O.apx_evd_ada(X, Om, 10)
    assert passes_evd == 5
    assert np.linalg.norm(X - (U * lam) @ U.T) / np.linalg.norm(X) < 1e-12
    # a slowly decaying spectrum keeps improving by more than tol for a while
    rng = np.random.default_rng(24)
    V, _ = np.linalg.qr(rng.standard_normal((300, 300)))
    Xs = (V * (1.0 / (1.0 + np.arange(300)) ** 0.5)) @ V.T
    _, hs, _ = O.ada_rrf(Xs, rng.standard_normal((300, 12)), 10, tol=1e-3)
    assert all(a - b >= 1e-3 for a, b in zip(hs[:-2], hs[1:-1]))
    assert len(hs) == 10 or hs[-2] - hs[-1] < 1e-3


def test_stop_rule_counts_consecutive_small_decreases():
    # residuals 1.0, 0.5, 0.4999, 0.49985, 0.3, 0.29995, 0.2999, 0.29989, 0.29988, ...: the run of
    # four small decreases starts after the jump to 0.3 (the one before it is broken)
    seq = iter([1.0, 0.5, 0.4999, 0.49985, 0.3, 0.29995, 0.2999, 0.29989, 0.29988, 0.2, 0.1])
    it, nr = O.stop_rule_phase(lambda: next(seq), 100, tol=1e-4, count=4)
    assert it == 9 and nr == 0.29988
    seq = iter([1.0, 0.9, 0.8])
    assert O.stop_rule_phase(lambda: next(seq), 3)[0] == 3  # the cap


def test_lai_schedule_reaches_the_full_solution_with_refinement():
    X, _ = _gmm(600, 3)
    rng = np.random.default_rng(31)
    Om = rng.standard_normal((600, 16))
    H0 = rng.random((600, 5)) * O.init_scale(X, 5)
    out = O.lai_schedule(X, Om, H0, O.default_alpha(X), q_max=6, max_iters=300, max_refine=300)
    W, H, _ = O.hals_symnmf(X, H0, O.default_alpha(X), 400, record=False)
    assert out["iters"] < 300 and out["checks"] >= 2
    assert out["nr_final"] <= O.normalized_residual(X, W, H) + 5e-3
