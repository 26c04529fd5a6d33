"""Pins for the oracle's warm-start network: finite differences, loss identity, Adam closed form."""

import numpy as np
import pytest

from oracle import mlp
from oracle import mlp as OM


def _net(seed=0):
    return mlp.init_params((6, 8, 7, 3), seed)


def test_gram_loss_matches_direct_outer_products():
    rng = np.random.default_rng(0)
    Hh, Hs = rng.random((25, 3)), rng.random((25, 3))
    L, _ = mlp.gram_loss(Hh, Hs)
    direct = np.linalg.norm(Hh @ Hh.T - Hs @ Hs.T) ** 2 / np.linalg.norm(Hs @ Hs.T) ** 2
    assert abs(L - direct) < 1e-12
    # column permutation of the target leaves the loss unchanged
    L2, _ = mlp.gram_loss(Hh, Hs[:, [2, 0, 1]])
    assert abs(L - L2) < 1e-12


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(1)
    params = _net()
    for p in params[1::2]:
        p += rng.normal(0, 0.1, size=p.shape)
    x = rng.standard_normal((30, 6))
    Hs = rng.random((30, 3))

    def loss(ps):
        out, _ = mlp.forward(ps, x)
        return mlp.gram_loss(out, Hs)[0]

    out, cache = mlp.forward(params, x)
    _, dH = mlp.gram_loss(out, Hs)
    grads = mlp.backward(params, cache, dH)
    eps = 1e-6
    for pi, (p, g) in enumerate(zip(params, grads)):
        flat = p.reshape(-1)
        for idx in rng.choice(flat.shape[0], size=min(6, flat.shape[0]), replace=False):
            old = flat[idx]
            flat[idx] = old + eps
            lp = loss(params)
            flat[idx] = old - eps
            lm = loss(params)
            flat[idx] = old
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - g.reshape(-1)[idx]) < 1e-6 + 1e-5 * abs(fd), (pi, idx)


def test_adam_first_step_closed_form():
    p = [np.array([1.0, -2.0, 3.0])]
    g = [np.array([0.5, -4.0, 1e-3])]
    m = [np.zeros(3)]
    v = [np.zeros(3)]
    mlp.adam_step(p, g, m, v, t=1, lr=0.01, eps=0.0)
    # with bias correction the first step is lr * sign(g)
    np.testing.assert_allclose(p[0], [0.99, -1.99, 2.99], rtol=1e-12)


def test_forward_nonnegative_output():
    x = np.random.default_rng(2).standard_normal((10, 6))
    out, _ = mlp.forward(_net(3), x)
    assert (out > 0).all()


def test_bf16_rounding_matches_torch_and_is_nearest_even():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(11)
    a = np.concatenate([rng.standard_normal(10000) * 10.0 ** rng.integers(-6, 6, 10000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.01171875, 3.0e38, -2.5e-30]])
    got = OM.round_bf16(a)
    ref = torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).double().numpy()
    np.testing.assert_array_equal(got, ref)
    # ties: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7 and goes to the even mantissa (1);
    # 1 + 3 * 2^-8 goes up to 1 + 2^-6
    assert OM.round_bf16(np.array([1.00390625]))[0] == 1.0
    assert OM.round_bf16(np.array([1.01171875]))[0] == 1.015625


def test_bf16_network_reduces_to_fp64_network_on_representable_values():
    # with x and every weight already bfloat16 values, the mixed-precision forward differs from the
    # FP64 one only through the rounding of the hidden activations
    rng = np.random.default_rng(12)
    dims = (8, 16, 16, 4)
    params = [OM.round_bf16(p) for p in OM.init_params(dims, 3)]
    x = OM.round_bf16(rng.standard_normal((20, 8)))
    y64, _ = OM.forward(params, x)
    y16, _ = OM.forward(params, x, bf16=True)
    assert np.abs(y16 - y64).max() < 2e-2 * np.abs(y64).max()
    assert not np.array_equal(y16, y64)
