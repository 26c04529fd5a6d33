"""FP64 oracle for the warm-start network (TEST INFRASTRUCTURE ONLY).

The network maps a node's normalised sketch row x_i = (X Omega)_i / ||(X Omega)_i||
(Omega from the range finder of Alg. RRF) to a nonnegative starting row of H:

    a1 = relu(x W1 + b1),  a2 = relu(a1 W2 + b2),  H0 = softplus(a2 W3 + b3).

Loss (invariant to permuting the columns of H): with H^ the network output
for all n rows of one instance and H* a converged SymNMF factor of it,

    L = ||H^ H^^T - H* H*^T||_F^2 / ||H* H*^T||_F^2
      = (||H^^T H^||^2 - 2 ||H^^T H*||^2 + ||H*^T H*||^2) / ||H*^T H*||^2,

evaluated with k x k Grams only.  dL/dH^ = 4 (H^ (H^^T H^) - H* (H*^T H^)) / ||H*^T H*||^2.

The paper initialises H uniformly at random (experiments section); this
network is an addition, so its parity is pinned only by finite differences.
"""

from __future__ import annotations

import numpy as np


def init_params(dims, seed):
    """He-uniform weights, zero biases; dims = (in, h1, h2, out)."""
    rng = np.random.default_rng(seed)
    params = []
    for a, b in zip(dims[:-1], dims[1:]):
        lim = np.sqrt(6.0 / a)
        params.append(rng.uniform(-lim, lim, size=(a, b)))
        params.append(np.zeros(b))
    return params


def round_bf16(a):
    """Round to bfloat16 (8-bit mantissa), nearest-even on the 16 dropped bits of the float32 value.

    The library's tensor-core products take their operands in this format: the mixed-precision
    network below rounds exactly those operands, so that its products agree with the GPU's FP32
    accumulation of the same BF16 values.
    """
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    keep = (b >> np.uint64(16)) & np.uint64(1)
    r = ((b + np.uint64(0x7FFF) + keep) >> np.uint64(16)) << np.uint64(16)
    return (r & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32).astype(np.float64)


def _q(a, bf16):
    """An operand of a product: itself, or (float32 then) bfloat16 when `bf16`."""
    if not bf16:
        return a
    return round_bf16(np.asarray(a, dtype=np.float64).astype(np.float32))


def softplus(z):
    return np.logaddexp(0.0, z)


def sigmoid(z):
    return 0.5 * (1.0 + np.tanh(0.5 * z))


def forward(params, x, bf16=False):
    """Network output and the cache of the backward pass.  With `bf16`, the operands of the three
    products (x, a1, a2 and W1, W2, W3) are rounded to bfloat16; the rest stays FP64."""
    W1, b1, W2, b2, W3, b3 = params
    z1 = _q(x, bf16) @ _q(W1, bf16) + b1
    a1 = np.maximum(z1, 0.0)
    z2 = _q(a1, bf16) @ _q(W2, bf16) + b2
    a2 = np.maximum(z2, 0.0)
    z3 = _q(a2, bf16) @ _q(W3, bf16) + b3
    return softplus(z3), (x, z1, a1, z2, a2, z3)


def gram_loss(Hhat, Hstar):
    """Column-permutation-invariant loss and its gradient with respect to Hhat."""
    A = Hhat.T @ Hhat
    B = Hhat.T @ Hstar
    C = Hstar.T @ Hstar
    norm = float((C * C).sum())
    L = (float((A * A).sum()) - 2.0 * float((B * B).sum()) + norm) / norm
    dH = 4.0 * (Hhat @ A - Hstar @ B.T) / norm
    return L, dH


def backward(params, cache, dout, bf16=False):
    """Gradients of sum(dout * H0) with respect to all parameters.  With `bf16`, the operands of
    the five backward products (activations, pre-activation gradients, weights) are rounded to
    bfloat16, as the library's tensor-core backward pass takes them."""
    W1, b1, W2, b2, W3, b3 = params
    x, z1, a1, z2, a2, z3 = cache
    q = lambda a: _q(a, bf16)  # noqa: E731
    dz3 = dout * sigmoid(z3)
    dW3 = q(a2).T @ q(dz3)
    db3 = dz3.sum(0)
    da2 = q(dz3) @ q(W3).T
    dz2 = da2 * (z2 > 0)
    dW2 = q(a1).T @ q(dz2)
    db2 = dz2.sum(0)
    da1 = q(dz2) @ q(W2).T
    dz1 = da1 * (z1 > 0)
    dW1 = q(x).T @ q(dz1)
    db1 = dz1.sum(0)
    return [dW1, db1, dW2, db2, dW3, db3]


def adam_step(params, grads, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015) in place; t counts from 1."""
    for p, g, mm, vv in zip(params, grads, m, v):
        mm *= b1
        mm += (1 - b1) * g
        vv *= b2
        vv += (1 - b2) * g * g
        mhat = mm / (1 - b1 ** t)
        vhat = vv / (1 - b2 ** t)
        p -= lr * mhat / (np.sqrt(vhat) + eps)


def sketch_features(XOmega):
    """Row-normalised sketch rows x_i = (X Omega)_i / ||(X Omega)_i||."""
    nrm = np.linalg.norm(XOmega, axis=1, keepdims=True)
    return XOmega / np.maximum(nrm, 1e-30)
