"""GPU parity of the warm-start network: forward, loss and gradients against the FP64 oracle.

Every product on the GPU is a BF16 x BF16 tensor-core GEMM with FP32 accumulation; the oracle's
mixed-precision form (`bf16=True`) rounds exactly the same operands to bfloat16 and keeps the
rest in FP64, so the two differ only by accumulation order and the rare operand whose FP32 and
FP64 values round to different bfloat16 neighbours."""

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
    ref, cache = OM.forward(params, x.astype(np.float32).astype(np.float64), bf16=True)
    # An activation whose FP32 (GPU) and FP64 (oracle) values straddle a bfloat16 rounding
    # boundary rounds to different neighbours: one term of a 256-term sum then moves by one
    # bfloat16 step, 2^-8 |a| |w|.  Nearly every output is untouched; the rest stay within a few
    # such steps.
    err = np.abs(got - ref)
    ok = err <= 1e-5 + 1e-4 * np.abs(ref)
    assert ok.mean() > 0.99, ok.mean()
    a2 = cache[4]
    step = 2.0 ** -8 * np.abs(a2).max() * np.abs(params[4]).max()
    assert err.max() <= 4 * step, (err.max(), step)
    # and the FP64 network is within BF16 operand rounding of both
    full, _ = OM.forward(params, x.astype(np.float32).astype(np.float64))
    assert np.abs(got - full).max() < 2e-2 * np.abs(full).max()


def _exact_network(rng, dims, rows):
    """Inputs and weights on small dyadic grids: every operand is exact in bfloat16 and every
    partial sum of every product is exact in float32, whatever the order of accumulation, so the
    GPU's products equal the oracle's and both round the same activations to bfloat16."""
    d0, d1, d2, d3 = dims
    x = rng.integers(-2, 3, size=(rows, d0)) / 4.0
    W1 = rng.integers(-2, 3, size=(d0, d1)) / 8.0
    b1 = rng.integers(-8, 9, size=d1) / 32.0
    W2 = rng.integers(-1, 2, size=(d1, d2)) / 8.0
    b2 = rng.integers(-8, 9, size=d2) / 256.0
    W3 = rng.integers(-1, 2, size=(d2, d3)) / 8.0
    b3 = rng.integers(-8, 9, size=d3) / 2048.0
    params = [W1, b1, W2, b2, W3, b3]
    _, cache = OM.forward(params, x, bf16=True)
    a1q, a2q = OM.round_bf16(cache[2]), OM.round_bf16(cache[4])
    # exactness: grids 1/32, 1/256, 1/2048 and bounds on |partial sums| below 2^24 grid steps
    assert np.all(np.abs(x) @ np.abs(W1) < 2.0 ** 24 / 32)
    assert np.all(np.abs(a1q) @ np.abs(W2) < 2.0 ** 24 / 256)
    assert np.all(np.abs(a2q) @ np.abs(W3) < 2.0 ** 24 / 2048)
    assert np.all(a1q * 32 == np.round(a1q * 32)) and np.all(a2q * 256 == np.round(a2q * 256))
    return x, params


@pytest.mark.parametrize("rows,dims", [(777, (74, 256, 256, 32)), (130, (20, 100, 300, 17))])
def test_forward_exact_on_dyadic_network(S, rows, dims):
    rng = np.random.default_rng(rows)
    x, params = _exact_network(rng, dims, rows)
    net = S.MLP(dims, seed=0)
    net.set_params(np.concatenate([p.ravel() for p in params]).astype(np.float32))
    got = np64(net.forward(t32(x)))
    ref, cache = OM.forward(params, x, bf16=True)
    # z3 is exact on both sides; only softplus differs (float32 on the GPU)
    np.testing.assert_allclose(got, ref, rtol=2e-6, atol=1e-7)
    # the pin has teeth: a transposed operand or a dropped bias moves the output far more
    wrong, _ = OM.forward([params[0], 0 * params[1]] + params[2:], x, bf16=True)
    assert np.abs(wrong - ref).max() > 1e-3


def test_init_is_he_uniform(S):
    net, _, _ = _net_and_data(S, seed=3)
    W1, b1, W2, b2, W3, b3 = net.unflatten(net.params())
    assert np.abs(W1).max() <= np.sqrt(6 / 74) and np.abs(W2).max() <= np.sqrt(6 / 256)
    assert abs(W2.std() - np.sqrt(6 / 256) / np.sqrt(3)) < 0.01
    assert not b1.any() and not b2.any() and not b3.any()


@pytest.mark.parametrize(
    "rows,dims",
    [(777, (74, 256, 256, 32)), (20000, (74, 256, 256, 32)), (5, (20, 100, 300, 17)), (3001, (9, 40, 512, 64))],
)
def test_loss_and_gradients_match_oracle(S, rows, dims):
    net, x, Hs = _net_and_data(S, rows=rows, dims=dims, seed=rows)
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
    out, cache = OM.forward(params, x64, bf16=True)
    L, dH = OM.gram_loss(out, H64)
    grads = OM.backward(params, cache, dH, bf16=True)
    assert loss == pytest.approx(L, rel=1e-4)
    gg = net.unflatten(np64(g))
    for a, b in zip(gg, grads):
        scale = np.abs(b).max() + 1e-12
        assert np.abs(a - b).max() / scale < 5e-4


def test_adam_training_lowers_loss(S):
    net, x, Hs = _net_and_data(S, rows=4000, seed=5)
    xt, Ht = t32(x), t32(Hs)
    l0 = net.loss_grad(xt, Ht)
    for _ in range(150):
        net.loss_grad(xt, Ht)
        net.adam(1e-3)
    assert net.loss_grad(xt, Ht) < 0.5 * l0
