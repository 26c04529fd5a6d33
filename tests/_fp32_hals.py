"""A float32 numpy restatement of the regularised HALS sweep (Eq. symhals_update2).

Test helper, not part of the oracle: it runs the oracle's sweep in float32
arithmetic (products, Grams and column updates all float32, objective by the
direct formula in float64) to show how far any float32 arithmetic drifts from
the FP64 oracle on a given instance.  A GPU deviation within a small multiple of
this drift is trajectory sensitivity of the iteration, not a kernel error.
"""

import numpy as np


def _half(Fu, Ff, Y, G, alpha):
    a = np.float32(alpha)
    for i in range(Fu.shape[1]):
        hh = G[i, i]
        r = Y[:, i] - Fu @ G[:, i] + a * Ff[:, i]
        Fu[:, i] = np.maximum(r / (hh + a) + hh / (hh + a) * Fu[:, i], np.float32(0))
    return Fu


def hals_fp32(X, H0, alpha, sweeps):
    """(W, H, objs): `sweeps` float32 sweeps from W0 = H0; objs in float64 from the float32 factors."""
    X32 = np.asarray(X, dtype=np.float32)
    H = np.array(H0, dtype=np.float32)
    W = H.copy()
    objs = []
    for _ in range(sweeps):
        W = _half(W, H, X32 @ H, H.T @ H, alpha)
        H = _half(H, W, X32 @ W, W.T @ W, alpha)
        Wd, Hd = W.astype(np.float64), H.astype(np.float64)
        R = np.asarray(X, dtype=np.float64) - Wd @ Hd.T
        objs.append(float((R * R).sum() + alpha * ((Wd - Hd) ** 2).sum()))
    return W.astype(np.float64), H.astype(np.float64), objs
