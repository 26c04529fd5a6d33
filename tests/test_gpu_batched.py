"""GPU parity of the batched grouped solver (many problems, stacked restarts, one grouped launch)."""

import numpy as np
import pytest
import torch

from oracle import philox
from oracle import symnmf as O
from synth import batched_problem_specs, dense_sbm

from ._gpu_util import np64, rel_err

pytestmark = pytest.mark.gpu

SPECS = [(200, 8), (513, 12), (1000, 16), (777, 24), (67, 32), (1500, 8)]


def _problems(dtype):
    Xs, Xn = [], []
    for p, (n, k) in enumerate(SPECS):
        A, _ = dense_sbm(n, k, seed=100 + p)
        Xn.append(A.astype(np.float64))
        t = torch.tensor(A, device="cuda")
        if dtype == torch.bfloat16:
            ld = (n + 7) // 8 * 8
            buf = torch.zeros((n, ld), dtype=torch.bfloat16, device="cuda")
            buf[:, :n] = t.to(torch.bfloat16)
            Xs.append(buf)
        else:
            Xs.append(t)
    return Xs, Xn


def _batch(S, Xs, R=4):
    # the binding takes X's row count as n and its row pitch as ldx
    return S.Batch(Xs, [k for _, k in SPECS], restarts=R, seeds=[7 * p + 1 for p in range(len(SPECS))])


def test_batched_init_is_per_restart_philox(S):
    Xs, Xn = _problems(torch.float32)
    b = _batch(S, Xs)
    b.init_random(scaled=True)
    for p, (n, k) in enumerate(SPECS):
        H, W = (np64(t) for t in b.factors(p))
        for r in range(4):
            ref = philox.philox_uniform_factor(n, k, 7 * p + 1 + r) * O.init_scale(Xn[p], k)
            np.testing.assert_allclose(H[:, r * k:(r + 1) * k], ref.astype(np.float32), rtol=1e-6)
        np.testing.assert_array_equal(H, W)


def test_batched_fp32_matches_oracle_per_restart(S):
    Xs, Xn = _problems(torch.float32)
    b = _batch(S, Xs)
    b.init_random(scaled=True)
    H0 = [np64(b.factors(p)[0]) for p in range(len(SPECS))]
    obj = b.sweep(25)
    for p, (n, k) in enumerate(SPECS):
        for r in range(4):
            Hi = H0[p][:, r * k:(r + 1) * k]
            _, _, ref = O.hals_symnmf(Xn[p], Hi, O.default_alpha(Xn[p]), 25)
            got = obj[:, p * 4 + r]
            assert rel_err(got, ref).max() < 1e-4, (p, r)


def test_batched_bf16_grouped_launch_reaches_oracle_residual(S):
    Xs, Xn = _problems(torch.bfloat16)
    b = _batch(S, Xs)
    b.init_random(scaled=True)
    H0 = [np64(b.factors(p)[0]) for p in range(len(SPECS))]
    b.sweep(40, record=False)
    info = b.info()
    assert info["stages"] in (3, 4, 6) and info["product_ms"] > 0
    for p, (n, k) in enumerate(SPECS):
        H, W = (np64(t) for t in b.factors(p))
        for r in range(4):
            c = slice(r * k, (r + 1) * k)
            Wo, Ho, _ = O.hals_symnmf(Xn[p], H0[p][:, c], O.default_alpha(Xn[p]), 40, record=False)
            nr_gpu = O.normalized_residual(Xn[p], W[:, c], H[:, c])
            nr_ref = O.normalized_residual(Xn[p], Wo, Ho)
            assert abs(nr_gpu - nr_ref) < 1e-3, (p, r, nr_gpu, nr_ref)


def test_batched_objectives_monotone_and_graph_replay(S):
    # FP32 products: monotone up to FP32 rounding of the trace-trick terms
    Xs, Xn = _problems(torch.float32)
    b = _batch(S, Xs, R=2)
    b.init_random(scaled=True)
    obj = b.sweep(30)
    nx = np.array([(X * X).sum() for X in Xn for _ in range(2)])
    assert (np.diff(obj, axis=0) <= 1e-7 * nx).all()
    n0 = S.launch_count()
    b.sweep(10, record=False)
    assert S.launch_count() > n0  # graph replays are counted per kernel node


@pytest.mark.gpu
def test_batched_spec_generator_shapes():
    specs = batched_problem_specs(64, seed=0)
    assert len(specs) == 64
    assert all(500 <= s["n"] <= 8000 and s["k"] in (8, 12, 16, 24, 32) for s in specs)
