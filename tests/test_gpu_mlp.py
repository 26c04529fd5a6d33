"""GPU parity of the warm-start network: forward, loss and gradients against the FP64 oracle."""

import numpy as np
import pytest
import torch

from oracle import mlp as OM

from ._gpu_util import np64, t32

pytestmark = pytest.mark.gpu


def _net_and_data(S, rows=3000, dims=(74, 256, 256, 32), seed=0):
    net = S.MLP(dims, seed=seed)
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((rows, dims[0]))
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    Hs = rng.random((rows, dims[3])) * 0.3
    return net, x, Hs


def test_forward_matches_oracle(S):
    net, x, _ = _net_and_data(S)
    params = [p.astype(np.float64) for p in net.unflatten(net.params())]
    got = np64(net.forward(t32(x)))
    ref, _ = OM.forward(params, x.astype(np.float32).astype(np.float64))
    np.testing.assert_allclose(got, ref, rtol=1e-4, atol=1e-5)


def test_init_is_he_uniform(S):
    net, _, _ = _net_and_data(S, seed=3)
    W1, b1, W2, b2, W3, b3 = net.unflatten(net.params())
    assert np.abs(W1).max() <= np.sqrt(6 / 74) and np.abs(W2).max() <= np.sqrt(6 / 256)
    assert abs(W2.std() - np.sqrt(6 / 256) / np.sqrt(3)) < 0.01
    assert not b1.any() and not b2.any() and not b3.any()


@pytest.mark.parametrize("rows", [777, 20000])
def test_loss_and_gradients_match_oracle(S, rows):
    net, x, Hs = _net_and_data(S, rows=rows, seed=rows)
    # non-zero biases so that every gradient path is exercised
    flat = net.params()
    rng = np.random.default_rng(1)
    P = net.unflatten(flat)
    for b in P[1::2]:
        b += rng.normal(0, 0.05, size=b.shape).astype(np.float32)
    net.set_params(flat)
    loss, g = net.loss_grad(t32(x), t32(Hs), want_grads=True)
    params = [p.astype(np.float64) for p in net.unflatten(net.params())]
    x64 = x.astype(np.float32).astype(np.float64)
    H64 = Hs.astype(np.float32).astype(np.float64)
    out, cache = OM.forward(params, x64)
    L, dH = OM.gram_loss(out, H64)
    grads = OM.backward(params, cache, dH)
    assert loss == pytest.approx(L, rel=1e-4)
    gg = net.unflatten(np64(g))
    for a, b in zip(gg, grads):
        scale = np.abs(b).max() + 1e-12
        assert np.abs(a - b).max() / scale < 2e-3


def test_adam_training_lowers_loss(S):
    net, x, Hs = _net_and_data(S, rows=4000, seed=5)
    xt, Ht = t32(x), t32(Hs)
    l0 = net.loss_grad(xt, Ht)
    for _ in range(150):
        net.loss_grad(xt, Ht)
        net.adam(1e-3)
    assert net.loss_grad(xt, Ht) < 0.5 * l0
