"""Further pins of oracle functions that feed other pins: ARI, the projected-gradient mask,
and the Philox counters of LvS-SymNMF's draws."""

import numpy as np
import pytest

from oracle import philox
from oracle import symnmf as O


def test_adjusted_rand_index_known_values():
    # Hubert & Arabie's index on a 6-point example worked by hand: contingency table
    # [[2, 1, 0], [0, 1, 2]]: sum C(n_ij, 2) = 2, row term 6, column term 3, C(6, 2) = 15,
    # expected 6 * 3 / 15 = 1.2, max (6 + 3) / 2 = 4.5, ARI = 0.8 / 3.3 = 8 / 33
    a = [0, 0, 0, 1, 1, 1]
    b = [0, 0, 1, 1, 2, 2]
    assert O.adjusted_rand_index(a, b) == pytest.approx(8.0 / 33.0, rel=1e-14)
    # symmetric and invariant to renaming the labels
    assert O.adjusted_rand_index(b, a) == pytest.approx(8.0 / 33.0, rel=1e-14)
    assert O.adjusted_rand_index([5, 5, 5, 9, 9, 9], [7, 7, 3, 3, 1, 1]) == pytest.approx(8.0 / 33.0, rel=1e-14)
    # a perfect match is 1; two labelings of 2 x 2 crossed blocks have index -1/2
    assert O.adjusted_rand_index([0, 0, 1, 1], [1, 1, 0, 0]) == 1.0
    assert O.adjusted_rand_index([0, 0, 1, 1], [0, 1, 0, 1]) == pytest.approx(-0.5, rel=1e-14)


def test_adjusted_rand_index_matches_library_and_vanishes_on_independent_labels():
    sk = pytest.importorskip("sklearn.metrics")
    rng = np.random.default_rng(0)
    for _ in range(20):
        a = rng.integers(0, 5, size=200)
        b = np.where(rng.random(200) < 0.6, a, rng.integers(0, 7, size=200))
        assert O.adjusted_rand_index(a, b) == pytest.approx(sk.adjusted_rand_score(a, b), rel=1e-12, abs=1e-14)
    # independent labelings: expectation 0, standard deviation ~ 1e-3 at this size
    a = rng.integers(0, 10, size=20000)
    b = rng.integers(0, 10, size=20000)
    assert abs(O.adjusted_rand_index(a, b)) < 5e-3


def test_projected_gradient_is_the_limit_of_the_projected_step():
    # ||grad^P f|| = lim_{t -> 0} ||P_+(Z - t grad f) - Z|| / t over Z = (W, H) (the projection onto
    # the nonnegative orthant).  The gradient here comes from central differences of the
    # surrogate objective, and the point has zeros with gradients of both signs: a mask that
    # dropped zero entries with a negative gradient (or kept those with a positive one) fails.
    rng = np.random.default_rng(5)
    n, k, alpha = 12, 3, 0.6
    A = rng.random((n, n))
    X = 0.5 * (A + A.T)
    W = rng.random((n, k))
    H = rng.random((n, k))
    W[::3, 0] = 0.0
    H[1::4, 2] = 0.0

    def fd_grad(M, which):
        g = np.zeros_like(M)
        h = 1e-6
        for idx in np.ndindex(M.shape):
            Mp, Mm = M.copy(), M.copy()
            Mp[idx] += h
            Mm[idx] -= h
            if which == "W":
                fp, fm = O.surrogate_objective(X, Mp, H, alpha), O.surrogate_objective(X, Mm, H, alpha)
            else:
                fp, fm = O.surrogate_objective(X, W, Mp, alpha), O.surrogate_objective(X, W, Mm, alpha)
            g[idx] = (fp - fm) / (2 * h)
        return g

    gW, gH = fd_grad(W, "W"), fd_grad(H, "H")
    zeros_W = W == 0.0
    assert (gW[zeros_W] < 0).any() and (gW[zeros_W] > 0).any()
    t = 1e-9
    step = np.concatenate([(np.maximum(W - t * gW, 0.0) - W).ravel(), (np.maximum(H - t * gH, 0.0) - H).ravel()])
    limit = np.linalg.norm(step) / t
    assert O.projected_gradient_norm(X, W, H, alpha) == pytest.approx(limit, rel=1e-6)


def test_lvs_symnmf_draws_use_iteration_and_side_counters():
    # the W-half of iteration t draws with Philox counter (j, t, 0, 3), the H-half with (j, t, 1, 3):
    # the traced random indices must be the first rows whose inclusive integer CDF exceeds
    # floor(u_j T / 2^64) for exactly those words
    rng = np.random.default_rng(9)
    n, k, s, tau, seed = 400, 4, 60, 1.0, 77
    A = (rng.random((n, n)) < 0.05).astype(float)
    X = np.maximum(A, A.T) + np.eye(n)
    H0 = rng.random((n, k))
    trace = []
    O.lvs_symnmf(X, H0, 1.0, 3, s, tau, seed, trace=trace)
    assert [side for side, _ in trace] == ["W", "H"] * 3
    for pos, (_, smp) in enumerate(trace):
        it, side = pos // 2, pos % 2
        words = philox.philox_sample_words(smp["s_R"], it, side, seed)
        C, T = smp["C"], smp["T"]
        expect = [int(np.searchsorted(C, np.uint64((w * T) >> 64), side="right")) for w in words]
        got = list(smp["idx"][smp["s_D"]:])
        assert got == expect
        # and they differ from the neighbouring counters' draws
        other = philox.philox_sample_words(smp["s_R"], it, 1 - side, seed)
        assert [int(np.searchsorted(C, np.uint64((w * T) >> 64), side="right")) for w in other] != got
