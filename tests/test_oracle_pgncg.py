"""Pins for the oracle's PGNCG / LAI-PGNCG (all-at-once Gauss-Newton for the SymNMF objective)."""

import numpy as np
import pytest

from oracle import symnmf as O
from synth import planted_dense


def _tiny(n=7, k=2, seed=0):
    rng = np.random.default_rng(seed)
    A = rng.random((n, n))
    return 0.5 * (A + A.T), rng.random((n, k))


def _explicit_jacobian(H):
    """Columns: d vec(H H^T) / d H_ij, by central differences (exact for a quadratic map)."""
    n, k = H.shape
    J = np.zeros((n * n, n * k))
    for c, idx in enumerate(np.ndindex(n, k)):
        E = np.zeros_like(H)
        E[idx] = 1.0
        J[:, c] = (((H + E) @ (H + E).T) - ((H - E) @ (H - E).T)).ravel() / 2.0
    return J


def test_jacobian_and_normal_operator_against_the_explicit_matrix():
    X, H = _tiny()
    J = _explicit_jacobian(H)
    rng = np.random.default_rng(1)
    P = rng.standard_normal(H.shape)
    np.testing.assert_allclose(O.gn_jacobian_apply(H, P).ravel(), J @ P.ravel(), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(O.gn_normal_apply(H, H.T @ H, P).ravel(), J.T @ (J @ P.ravel()),
                               rtol=1e-12, atol=1e-12)


def test_gradient_is_twice_j_transpose_r():
    # grad ||X - H H^T||^2 = 2 J^T r = 4 (H H^T - X) H, by central differences of the objective
    X, H = _tiny(seed=2)
    f = lambda M: float(((X - M @ M.T) ** 2).sum())  # noqa: E731
    g = np.zeros_like(H)
    for idx in np.ndindex(H.shape):
        E = np.zeros_like(H)
        E[idx] = 1e-6
        g[idx] = (f(H + E) - f(H - E)) / 2e-6
    R = 2.0 * (H @ (H.T @ H) - X @ H)  # J^T r as PGNCG forms it
    np.testing.assert_allclose(g, 2.0 * R, rtol=1e-6, atol=1e-8)


def test_cg_reaches_the_gauss_newton_step():
    # with as many CG steps as unknowns, Z solves min ||J z - r|| (J^T J is singular: the
    # rotations H -> H Q leave H H^T fixed; CG from 0 gives the minimum-norm solution)
    X, H = _tiny(n=6, k=2, seed=3)
    n, k = H.shape
    J = _explicit_jacobian(H)
    r = (H @ H.T - X).ravel()
    z_ls = np.linalg.lstsq(J, r, rcond=None)[0].reshape(n, k)
    Hn = O.pgncg_iteration(X @ H, H, s_max=n * k)
    np.testing.assert_allclose(Hn, np.maximum(H - z_ls, 0.0), rtol=1e-7, atol=1e-9)


def test_symnmf_objective_trace_trick():
    X, H = _tiny(n=9, k=3, seed=4)
    direct = float(((X - H @ H.T) ** 2).sum())
    assert O.symnmf_objective(float((X * X).sum()), H.T @ H, H.T @ X @ H) == pytest.approx(direct, rel=1e-12)


def test_pgncg_recovers_a_noiseless_planted_factor():
    X, H0, _ = planted_dense(n=200, k=4, sigma=0.0, seed=1)
    rng = np.random.default_rng(5)
    Hs = H0 + 0.05 * rng.random(H0.shape)  # start near the planted factor
    nx2 = float((X * X).sum())
    H, objs = O.pgncg_symnmf(lambda F: X @ F, nx2, Hs, 15, s_max=10)
    assert objs[-1] / nx2 < 1e-10
    assert objs[-1] < objs[0]


def test_lai_pgncg_equals_pgncg_when_the_range_is_captured():
    # rank(X) <= l: U Lambda U^T = X, so LAI-PGNCG iterates equal PGNCG iterates
    X, _, _ = planted_dense(n=150, k=5, sigma=0.0, seed=2)
    rng = np.random.default_rng(6)
    U, lam = O.apx_evd(X, rng.standard_normal((150, 12)), 1)
    H0 = rng.random((150, 5)) * O.init_scale(X, 5)
    nx2 = float((X * X).sum())
    Ha, oa = O.pgncg_symnmf(lambda F: X @ F, nx2, H0, 10)
    Hb, ob = O.pgncg_symnmf(lambda F: O.lai_product(U, lam, F), nx2, H0, 10)
    np.testing.assert_allclose(Hb, Ha, rtol=1e-8, atol=1e-10)
    np.testing.assert_allclose(ob, oa, rtol=1e-8)
