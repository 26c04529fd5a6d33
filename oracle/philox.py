"""Philox4x32-10 counter-based generator and the random streams built on it.

Written from the published definition (Salmon, Moraes, Dror, Shaw, "Parallel
random numbers: as easy as 1, 2, 3", SC'11): a 4 x 32-bit counter and a
2 x 32-bit key; each of the 10 rounds multiplies two counter words by fixed
constants, mixes the high/low halves with the other words and the key, and
then bumps the key by the Weyl constants.

Streams (each is a separate "tag" in counter word 3):

* TAG_OMEGA  - Gaussian test matrix, Box-Muller on two uniforms per call;
* TAG_INIT   - Uniform[0,1) starting factor;
* TAG_SAMPLE - 64-bit uniforms for hybrid leverage-score draws.

The CUDA path implements the same definition on its own; the two are
compared bit for bit on the integer outputs.
"""

from __future__ import annotations

import numpy as np

MASK32 = np.uint64(0xFFFFFFFF)
M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)

TAG_OMEGA = 1
TAG_INIT = 2
TAG_SAMPLE = 3


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10.  All inputs are array-likes of uint32 values.

    Returns four uint64 arrays holding the 32-bit output words.
    """
    c0 = np.asarray(c0, dtype=np.uint64) & MASK32
    c1 = np.asarray(c1, dtype=np.uint64) & MASK32
    c2 = np.asarray(c2, dtype=np.uint64) & MASK32
    c3 = np.asarray(c3, dtype=np.uint64) & MASK32
    k0 = np.asarray(k0, dtype=np.uint64) & MASK32
    k1 = np.asarray(k1, dtype=np.uint64) & MASK32
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    k0 = np.broadcast_to(k0, c0.shape).copy()
    k1 = np.broadcast_to(k1, c0.shape).copy()
    for rnd in range(10):
        p0 = M0 * c0  # < 2^64, exact in uint64
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0), lo1, (hi0 ^ c3 ^ k1), lo0
        if rnd != 9:
            k0 = (k0 + W0) & MASK32
            k1 = (k1 + W1) & MASK32
    return c0, c1, c2, c3


def _key(seed: int):
    return np.uint64(seed & 0xFFFFFFFF), np.uint64((seed >> 32) & 0xFFFFFFFF)


def philox_gaussian(n: int, l: int, seed: int) -> np.ndarray:
    """Gaussian test matrix Omega (n x l) from Philox + Box-Muller, float64.

    Entry pair (i, 2p), (i, 2p+1) comes from one call with counter
    (p, i mod 2^32, i >> 32, TAG_OMEGA) and key (seed_lo, seed_hi):
    u1 = (x0 + 1) / 2^32 in (0, 1], u2 = x1 / 2^32 in [0, 1),
    r = sqrt(-2 ln u1), z0 = r cos(2 pi u2), z1 = r sin(2 pi u2).
    """
    k0, k1 = _key(seed)
    npair = (l + 1) // 2
    i = np.repeat(np.arange(n, dtype=np.uint64), npair)
    p = np.tile(np.arange(npair, dtype=np.uint64), n)
    x0, x1, _, _ = philox4x32_10(p, i & MASK32, i >> np.uint64(32), TAG_OMEGA, k0, k1)
    u1 = (x0.astype(np.float64) + 1.0) * 2.0 ** -32
    u2 = x1.astype(np.float64) * 2.0 ** -32
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty((n, 2 * npair))
    z[:, 0::2] = (r * np.cos(2.0 * np.pi * u2)).reshape(n, npair)
    z[:, 1::2] = (r * np.sin(2.0 * np.pi * u2)).reshape(n, npair)
    return z[:, :l]


def philox_uniform_factor(n: int, k: int, seed: int) -> np.ndarray:
    """Uniform[0,1) factor: entry (i, j) = x0 / 2^32 with counter (j, i lo, i hi, TAG_INIT)."""
    k0, k1 = _key(seed)
    i = np.repeat(np.arange(n, dtype=np.uint64), k)
    j = np.tile(np.arange(k, dtype=np.uint64), n)
    x0, _, _, _ = philox4x32_10(j, i & MASK32, i >> np.uint64(32), TAG_INIT, k0, k1)
    return (x0.astype(np.float64) * 2.0 ** -32).reshape(n, k)


def philox_sample_words(count: int, it: int, side: int, seed: int) -> list[int]:
    """64-bit uniforms for draws j = 0..count-1 of iteration `it`, factor `side`.

    Counter (j, it, side, TAG_SAMPLE); the draw is u = x0 * 2^32 + x1.
    Returned as Python ints so that the 128-bit products stay exact.
    """
    if count <= 0:
        return []
    k0, k1 = _key(seed)
    j = np.arange(count, dtype=np.uint64)
    x0, x1, _, _ = philox4x32_10(j, it, side, TAG_SAMPLE, k0, k1)
    return [(int(a) << 32) | int(b) for a, b in zip(x0, x1)]
