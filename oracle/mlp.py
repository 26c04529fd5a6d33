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


def softplus(z):
    return np.logaddexp(0.0, z)


def sigmoid(z):
    return 0.5 * (1.0 + np.tanh(0.5 * z))


def forward(params, x):
    W1, b1, W2, b2, W3, b3 = params
    z1 = x @ W1 + b1
    a1 = np.maximum(z1, 0.0)
    z2 = a1 @ W2 + b2
    a2 = np.maximum(z2, 0.0)
    z3 = a2 @ W3 + b3
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


def backward(params, cache, dout):
    """Gradients of sum(dout * H0) with respect to all parameters."""
    W1, b1, W2, b2, W3, b3 = params
    x, z1, a1, z2, a2, z3 = cache
    dz3 = dout * sigmoid(z3)
    dW3 = a2.T @ dz3
    db3 = dz3.sum(0)
    da2 = dz3 @ W3.T
    dz2 = da2 * (z2 > 0)
    dW2 = a1.T @ dz2
    db2 = dz2.sum(0)
    da1 = dz2 @ W2.T
    dz1 = da1 * (z1 > 0)
    dW1 = x.T @ dz1
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
