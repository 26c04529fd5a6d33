"""Pins for the oracle's Compressed-SymNMF comparator (appendix, Compressed-NMF vs LAI-NMF)."""

import numpy as np
import pytest
import scipy.optimize as sopt

from oracle import symnmf as O
from synth import uniform_factor


def _problem(n=60, k=3, l=8, seed=0):
    rng = np.random.default_rng(seed)
    A = rng.random((n, n))
    X = 0.5 * (A + A.T)
    Q, _ = np.linalg.qr(X @ rng.standard_normal((n, l)))
    return X, Q, rng.random((n, k)), rng.random((n, k))


def test_bpp_half_is_the_exact_minimiser_of_the_compressed_problem():
    # min_{w_r >= 0} ||Q^T H w_r - Q^T x_r||^2 + alpha ||w_r - h_r||^2 row by row, solved as a stacked
    # nonnegative least-squares problem [Q^T H; sqrt(alpha) I] w = [Q^T x_r; sqrt(alpha) h_r]
    X, Q, W, H = _problem()
    alpha = 0.7
    Wn, _, _ = O.compressed_half(X.T @ Q, Q, W, H, alpha, rule="bpp")
    A = np.vstack([Q.T @ H, np.sqrt(alpha) * np.eye(3)])
    for r in range(X.shape[0]):
        b = np.concatenate([Q.T @ X[:, r], np.sqrt(alpha) * H[r]])
        w, _ = sopt.nnls(A, b)
        np.testing.assert_allclose(Wn[r], w, rtol=1e-8, atol=1e-10)


def test_hals_half_decreases_the_compressed_objective_and_full_basis_is_plain_hals():
    X, Q, W, H = _problem(seed=1)
    alpha = 0.5
    f = lambda Wm: float(((Q.T @ (H @ Wm.T - X)) ** 2).sum() + alpha * ((Wm - H) ** 2).sum())  # noqa: E731
    Wn, _, _ = O.compressed_half(X.T @ Q, Q, W, H, alpha)
    assert f(Wn) <= f(W)
    # Q = I: the compressed problem is the full one, so the sweeps are plain regularised HALS
    I = np.eye(X.shape[0])
    Wc, Hc, oc = O.compressed_symnmf(X, I, H, alpha, 5)
    Wf, Hf, of = O.hals_symnmf(X, H, alpha, 5)
    np.testing.assert_allclose(Hc, Hf, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(oc, of, rtol=1e-10)


def test_compressed_differs_from_lai_only_through_the_projected_gram():
    # the appendix's observation: both fit Q Q^T X.  For F in range(Q), the compressed right-hand
    # side X Q Q^T F projected onto range(Q) is the LAI one, Q Q^T X Q Q^T F, and the compressed
    # Gram F^T Q Q^T F is the LAI Gram F^T F
    X, Q, _, _ = _problem(seed=2)
    F = Q @ np.random.default_rng(3).random((Q.shape[1], 3))
    _, G_c, Y_c = O.compressed_half(X.T @ Q, Q, F, F, 1.0)
    lam, V = np.linalg.eigh(Q.T @ X @ Q)
    Y_lai = O.lai_product(Q @ V, lam, F)
    np.testing.assert_allclose(Q @ (Q.T @ Y_c), Y_lai, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(G_c, F.T @ F, rtol=1e-10, atol=1e-12)


def test_compressed_sweeps_are_monotone_in_each_half_objective():
    X, Q, _, H = _problem(n=80, k=4, l=12, seed=4)
    W, H2, objs = O.compressed_symnmf(X, Q, H, 1.0, 30)
    assert objs[-1] < objs[0]
    assert np.all(np.isfinite(objs))
