"""Error paths of the C ABI, provoked without faulting the GPU, and the FP64 Cholesky pins.

Each error is made on the host (a zero column, a NaN entry, a flag that nothing
sets); every device wait involved is bounded and returns a status the host reads.
"""

import numpy as np
import pytest
import torch

from synth import uniform_factor

from ._gpu_util import np64, t32, t64

pytestmark = pytest.mark.gpu


def _small_problem(S, n=300, k=6, seed=0, alpha=1.0):
    rng = np.random.default_rng(seed)
    A = rng.random((n, n))
    X = 0.5 * (A + A.T)
    return S.Solver(t32(X), k, alpha=alpha, seed=seed), X


def test_leverage_of_a_factor_with_a_zero_column_is_not_spd(S):
    # F^T F is singular when a column of F is zero: the FP64 Cholesky meets a zero pivot
    s, _ = _small_problem(S)
    H = uniform_factor(300, 6, seed=1)
    H[:, 3] = 0.0
    s.set_factors(t32(H))
    with pytest.raises(S.SymNMFError) as e:
        s.leverage(0)
    assert e.value.status == S.ENOTSPD
    # the handle stays usable: a full-rank factor gives leverage scores summing to k
    s.set_factors(t32(uniform_factor(300, 6, seed=2)))
    lev = np64(s.leverage(0))
    assert lev.sum() == pytest.approx(6.0, rel=1e-5)


def test_nonfinite_x_is_reported_at_create(S):
    rng = np.random.default_rng(3)
    A = rng.random((256, 256))
    X = 0.5 * (A + A.T)
    for bad in (np.nan, np.inf):
        Xb = X.copy()
        Xb[17, 40] = Xb[40, 17] = bad
        with pytest.raises(S.SymNMFError) as e:
            S.Solver(t32(Xb), 5, alpha=1.0, seed=4)
        assert e.value.status == S.ENAN
        # the same through the float32 copy of a BF16 problem
        with pytest.raises(S.SymNMFError) as e:
            S.Solver(t32(X).to(torch.bfloat16), 5, alpha=1.0, x_hi=t32(Xb))
        assert e.value.status == S.ENAN


def test_nan_in_the_operator_reaches_the_objective_and_is_reported(S):
    # a NaN eigenvalue given through set_lai: the recorded LAI objective is non-finite
    rng = np.random.default_rng(4)
    A = rng.random((256, 256))
    X = 0.5 * (A + A.T)
    Q, _ = np.linalg.qr(rng.standard_normal((256, 12)))
    lam = np.linspace(10.0, 1.0, 12)
    lam[5] = np.nan
    for mode in (0, 1):  # persistent engine, separate kernels
        s = S.Solver(t32(X), 5, alpha=1.0, seed=4, max_width=12, lai_mode=mode)
        s.set_lai(t32(Q), lam)
        s.set_factors(t32(uniform_factor(256, 5, seed=5)))
        with pytest.raises(S.SymNMFError) as e:
            s.sweep(2, source=S.SRC_LAI)
        assert e.value.status == S.ENAN


def test_nonfinite_or_negative_start_is_rejected(S):
    s, _ = _small_problem(S)
    H = uniform_factor(300, 6, seed=6)
    for bad in (np.nan, -0.5, np.inf):
        Hb = H.copy()
        Hb[10, 2] = bad
        with pytest.raises(S.SymNMFError) as e:
            s.set_factors(t32(Hb))
        assert e.value.status == S.EINVAL


def test_bounded_wait_runs_out_and_returns_timeout(S):
    s, X = _small_problem(S, n=200, k=4)
    st = S.symnmf_debug_wait_timeout(s.h, 2_000_000)  # 2 ms on a flag that nothing sets
    assert st == S.ETIMEOUT
    # the error word was cleared: the handle keeps working
    s.set_factors(t32(uniform_factor(200, 4, seed=7)))
    obj = s.sweep(3)
    assert np.all(np.isfinite(obj)) and obj[-1] <= obj[0]
    assert S.symnmf_debug_wait_timeout(s.h, 10) == S.EINVAL  # limits outside [1 us, 1 s]


def test_cholesky_of_an_indefinite_matrix_is_not_spd(S):
    G = np.diag([4.0, 1.0, -1.0, 2.0])
    with pytest.raises(S.SymNMFError) as e:
        S.cholesky(t64(G))
    assert e.value.status == S.ENOTSPD


def _gram_with_condition(k, cond, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((k, k)))
    s = np.logspace(0.0, -np.log10(cond), k)
    G = (Q * s) @ Q.T
    return 0.5 * (G + G.T)


@pytest.mark.parametrize("k", [20, 50, 64, 96])
@pytest.mark.parametrize("cond", [1e6, 1e9, 1e12])
def test_fp64_cholesky_is_backward_stable(S, k, cond):
    # Higham, Accuracy and Stability of Numerical Algorithms, Thm 10.3: the computed R of an
    # FP64 Cholesky satisfies |R^T R - G| <= gamma_{k+1} |R^T| |R| entrywise, gamma_m = m u / (1 - m u),
    # u = 2^-53.  A double-float (~2^-44) or FP32 factorisation would break this bound.
    u = 2.0 ** -53
    gam = lambda m: m * u / (1.0 - m * u)  # noqa: E731
    G = _gram_with_condition(k, cond, seed=k)
    R, Ri = S.cholesky(t64(G))
    R, Ri = np64(R), np64(Ri)
    assert np.all(np.tril(R, -1) == 0.0) and np.all(np.diag(R) > 0)
    bwd = np.abs(R.T @ R - G)
    bound = gam(k + 1) * (np.abs(R.T) @ np.abs(R))
    assert np.all(bwd <= 2.0 * bound), float((bwd / bound).max())
    # the inverse by row-wise back substitution: |R X - I| <= gamma_k |R| |X| (Higham, Sec. 14.2)
    res = np.abs(R @ Ri - np.eye(k))
    assert np.all(res <= 2.0 * gam(k) * (np.abs(R) @ np.abs(Ri)) + 1e-300)
    # against LAPACK's FP64 factor: within the first-order perturbation bound of the
    # Cholesky factor (Sun 1991), ||dR||_F / ||R||_2 <= kappa_2(G) ||dG||_F / ||G||_2 / sqrt(2),
    # for backward errors of size gamma_{k+1} ||G|| on both sides
    Rl = np.linalg.cholesky(G).T
    kap = np.linalg.cond(G)
    d = np.linalg.norm(R - Rl) / np.linalg.norm(Rl, 2)
    assert d <= 2.0 * kap * gam(k + 1) * np.sqrt(k) / np.sqrt(2.0)
    if cond <= 1e6:  # well conditioned: the two FP64 factors agree to ~1e-13
        assert d <= 1e-11
