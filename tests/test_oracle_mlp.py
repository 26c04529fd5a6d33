"""Pins for the oracle's warm-start network: finite differences, loss identity, Adam closed form."""

import numpy as np

from oracle import mlp


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
