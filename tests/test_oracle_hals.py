"""Pins for the oracle's HALS / BPP updates, objectives and convergence claims."""

import numpy as np
import pytest

from oracle import symnmf as O
from synth import planted_dense, uniform_factor


def _small(n=40, k=4, seed=0):
    rng = np.random.default_rng(seed)
    A = rng.random((n, n))
    X = 0.5 * (A + A.T)
    H = rng.random((n, k))
    W = rng.random((n, k))
    return X, W, H


@pytest.mark.parametrize("alpha", [0.0, 0.3, 2.0])
def test_efficient_rule_equals_explicit_residual_rule(alpha):
    # Eq. symhals_update2 is an algebraic rewrite of Eq. symhals_update1
    X, W, H = _small()
    if alpha == 0.0:
        alpha = 1e-9
    G, Y = H.T @ H, X @ H
    a = O.hals_update_efficient(W, H, G, Y, alpha)
    b = O.hals_update_explicit(X, W, H, alpha)
    np.testing.assert_allclose(a, b, rtol=1e-11, atol=1e-12)


def test_regularised_equals_standard_hals_on_shifted_gram():
    # Update(G + alpha I, Y + alpha H) with the standard rule == regularised rule
    X, W, H = _small(seed=1)
    alpha = 0.7
    k = H.shape[1]
    G, Y = H.T @ H, X @ H
    a = O.hals_update_efficient(W, H, G, Y, alpha)
    b = O.hals_update_standard(W, G + alpha * np.eye(k), Y + alpha * H)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)


def test_alpha_zero_is_plain_hals():
    X, W, H = _small(seed=2)
    G, Y = H.T @ H, X @ H
    a = O.hals_update_efficient(W, H, G, Y, 0.0)
    b = O.hals_update_standard(W, G, Y)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)


def test_each_column_update_is_the_exact_block_minimiser():
    # KKT of min_{w_i >= 0} f(W, H): g = 0 where w_i > 0, g >= 0 where w_i = 0
    X, W, H = _small(n=30, k=5, seed=3)
    alpha = 0.4
    G, Y = H.T @ H, X @ H
    Wn = W.copy()
    for i in range(5):
        Wn = O.hals_update_efficient(Wn, H, G, Y, alpha) if i == 0 else Wn
    # check column optimality for the final W with the other columns fixed
    for i in range(5):
        g = 2.0 * (Wn @ G[:, i] - Y[:, i]) + 2.0 * alpha * (Wn[:, i] - H[:, i])
        # after the full column sweep, column k-1 is exactly optimal; earlier ones
        # were optimal w.r.t. the then-current later columns, so test the last one
        if i == 4:
            pos = Wn[:, i] > 0
            assert np.abs(g[pos]).max() < 1e-9
            assert (g[~pos] > -1e-9).all()


def test_objective_non_increasing_per_column_update():
    X, W, H = _small(n=35, k=6, seed=4)
    alpha = 1.0
    G, Y = H.T @ H, X @ H
    f0 = O.surrogate_objective(X, W, H, alpha)
    Wc = W.copy()
    for i in range(6):
        # update only column i with the efficient formula
        hh = G[i, i]
        r = Y[:, i] - Wc @ G[:, i] + alpha * H[:, i]
        Wc[:, i] = np.maximum(r / (hh + alpha) + hh / (hh + alpha) * Wc[:, i], 0.0)
        f1 = O.surrogate_objective(X, Wc, H, alpha)
        assert f1 <= f0 + 1e-10 * abs(f0)
        f0 = f1


def test_trace_trick_equals_direct_residual():
    X, W, H = _small(seed=5)
    direct = np.linalg.norm(X - W @ H.T) ** 2
    tt = O.trace_trick_residual_sq((X * X).sum(), W.T @ W, H.T @ H, W.T @ X @ H)
    assert abs(direct - tt) <= 1e-10 * direct


@pytest.mark.parametrize("rule", ["hals", "bpp"])
def test_monotone_surrogate_on_planted(rule):
    X, H0, _ = planted_dense(n=200, k=4, sigma=0.01, seed=0)
    alpha = O.default_alpha(X)
    Hi = uniform_factor(200, 4, seed=0)
    _, _, objs = O.hals_symnmf(X, Hi, alpha, 15 if rule == "bpp" else 40, rule=rule)
    d = np.diff(objs)
    assert (d <= 1e-10 * np.abs(np.array(objs[:-1]))).all()


def test_projected_gradient_matches_finite_differences():
    X, W, H = _small(n=12, k=3, seed=6)
    alpha = 0.8
    f = lambda W_, H_: O.surrogate_objective(X, W_, H_, alpha)  # noqa: E731
    gW = 2.0 * (W @ (H.T @ H) - X @ H) + 2.0 * alpha * (W - H)
    eps = 1e-6
    for (r, c) in [(0, 0), (5, 2), (11, 1)]:
        Wp, Wm = W.copy(), W.copy()
        Wp[r, c] += eps
        Wm[r, c] -= eps
        fd = (f(Wp, H) - f(Wm, H)) / (2 * eps)
        assert abs(fd - gW[r, c]) < 1e-5 * max(1.0, abs(fd))
    # all variables strictly positive -> projected gradient is the full gradient
    gH = 2.0 * (H @ (W.T @ W) - X @ W) + 2.0 * alpha * (H - W)
    pg = O.projected_gradient_norm(X, W, H, alpha)
    assert abs(pg - np.sqrt((gW ** 2).sum() + (gH ** 2).sum())) < 1e-10 * pg


def test_kkt_residual_vanishes_at_convergence():
    X, _, _ = planted_dense(n=300, k=3, sigma=0.01, seed=1)
    alpha = O.default_alpha(X)
    Hi = uniform_factor(300, 3, seed=1)
    W, H, _ = O.hals_symnmf(X, Hi, alpha, 400, record=False)
    pg0 = O.projected_gradient_norm(X, Hi, Hi, alpha)
    pg = O.projected_gradient_norm(X, W, H, alpha)
    assert pg / pg0 < 1e-6


@pytest.mark.slow
def test_exact_recovery_on_noiseless_planted():
    X, H0, labels = planted_dense(n=1000, k=10, sigma=0.0, seed=0)
    alpha = O.default_alpha(X)
    ok = False
    # the experiments' start: Uniform[0,1] scaled by 2 sqrt(mean(X) / k); an
    # unscaled start zeroes most columns in the first sweep (a poor local minimum)
    for seed in range(4):
        Hi = uniform_factor(1000, 10, seed=seed) * O.init_scale(X, 10)
        W, H, _ = O.hals_symnmf(X, Hi, alpha, 600, record=False)
        nr = O.normalized_residual(X, W, H)
        if nr < 1e-4:
            assert O.adjusted_rand_index(O.cluster_labels(H), labels) == 1.0
            ok = True
            break
    assert ok


def test_noisy_planted_reaches_noise_floor():
    X, H0, labels = planted_dense(n=1000, k=10, sigma=0.01, seed=0)
    alpha = O.default_alpha(X)
    Xc = H0 @ H0.T
    floor = np.linalg.norm(X - Xc) / np.linalg.norm(X)
    best = 1.0
    for seed in range(3):
        Hi = uniform_factor(1000, 10, seed=seed) * O.init_scale(X, 10)
        W, H, _ = O.hals_symnmf(X, Hi, alpha, 300, record=False)
        best = min(best, O.normalized_residual(X, W, H))
    assert best <= floor + 1e-3


def test_nls_rows_match_bruteforce():
    rng = np.random.default_rng(7)
    for k in (2, 5, 8):
        A = rng.standard_normal((3 * k, k))
        Gp = A.T @ A + 0.1 * np.eye(k)
        Y = rng.standard_normal((6, k))
        got = O.nls_rows(Gp, Y)
        for r in range(6):
            ref = O.nls_row_bruteforce(Gp, Y[r])
            np.testing.assert_allclose(got[r], ref, rtol=1e-8, atol=1e-10)


def test_nls_rows_satisfy_kkt():
    rng = np.random.default_rng(8)
    k = 10
    A = rng.standard_normal((40, k))
    Gp = A.T @ A + 0.5 * np.eye(k)
    Y = rng.standard_normal((20, k)) * 3
    X = O.nls_rows(Gp, Y)
    g = X @ Gp - Y
    assert (X >= 0).all()
    assert np.abs(g[X > 0]).max() < 1e-8
    assert (g[X == 0] > -1e-8).all()
