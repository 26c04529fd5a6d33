"""Seeded generators for the five synthetic SymNMF workloads.

Every function here builds an *input*: a data matrix, a starting factor or a
Gaussian test matrix. Nothing here computes a step of the SymNMF method.

Workloads (sizes are the defaults the tests and the benchmark use):

* planted dense X = H0 H0^T + N, clipped at zero (n=1000, k=10, 10 blocks);
* Gaussian-mixture kernel matrices X_ij = exp(-||x_i - x_j||^2 / sigma^2),
  sigma the median pairwise distance (n=20000 in R^50, 20 components;
  n=50000 in R^64, 32 Dirichlet(1)-weighted components);
* stochastic-block-model graphs in CSR with unit weights and self loops
  (n=1e6, 64 equal communities, mean degree 30, p_in/p_out = 20);
* dense 0/1 SBM problems for the batched solver (n log-uniform in
  [500, 8000], k drawn from {8, 12, 16, 24, 32}).
"""

from __future__ import annotations

import math

import numpy as np

# ---------------------------------------------------------------- dense planted


def planted_dense(n: int = 1000, k: int = 10, sigma: float = 0.01, seed: int = 0,
                  lo: float = 0.5, hi: float = 1.0):
    """Planted block SymNMF instance.

    H0 has k disjoint row blocks of n/k rows; row i of block b carries a
    Uniform[lo, hi] entry in column b and zeros elsewhere.  N is symmetric
    Gaussian noise: the upper triangle (diagonal included) is drawn i.i.d.
    N(0, sigma^2) and mirrored.  X = max(H0 H0^T + N, 0), float64.

    Returns (X, H0, labels).
    """
    rng = np.random.default_rng(seed)
    labels = (np.arange(n) * k) // n
    H0 = np.zeros((n, k))
    H0[np.arange(n), labels] = rng.uniform(lo, hi, size=n)
    X = H0 @ H0.T
    if sigma > 0:
        N = rng.normal(0.0, sigma, size=(n, n))
        N = np.triu(N)
        N = N + np.triu(N, 1).T
        X = X + N
    np.maximum(X, 0.0, out=X)
    return X, H0, labels


def uniform_factor(n: int, k: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """Uniform[0, 1) starting factor (times `scale`), float64, n x k row-major."""
    rng = np.random.default_rng(seed + 0x5EED)
    return rng.random((n, k)) * scale


def gaussian_sketch(n: int, l: int, seed: int) -> np.ndarray:
    """Standard normal test matrix Omega (n x l), float64."""
    rng = np.random.default_rng(seed + 0x0E6A)
    return rng.standard_normal((n, l))


# ------------------------------------------------------- Gaussian-mixture kernel


def gmm_points(n: int, d: int, c: int, seed: int, weights: str = "equal",
               mean_std: float = 3.0):
    """Points from a c-component Gaussian mixture in R^d.

    Means ~ N(0, mean_std^2 I), unit covariance.  `weights` is "equal" or
    "dirichlet" (Dirichlet(1) mixing weights).  Returns (points float64 n x d,
    labels int64).
    """
    rng = np.random.default_rng(seed)
    means = rng.normal(0.0, mean_std, size=(c, d))
    if weights == "equal":
        w = np.full(c, 1.0 / c)
    elif weights == "dirichlet":
        w = rng.dirichlet(np.ones(c))
    else:
        raise ValueError(weights)
    labels = rng.choice(c, size=n, p=w)
    pts = means[labels] + rng.standard_normal((n, d))
    return pts, labels


def median_pair_distance(points: np.ndarray, seed: int, npairs: int = 1_000_000) -> float:
    """Median Euclidean distance over a fixed seeded sample of pairs i != j."""
    n = points.shape[0]
    rng = np.random.default_rng(seed + 0xD157)
    i = rng.integers(0, n, size=npairs)
    j = rng.integers(0, n - 1, size=npairs)
    j = j + (j >= i)  # j != i, uniform over the others
    dist = np.sqrt(((points[i] - points[j]) ** 2).sum(axis=1))
    return float(np.median(dist))


def kernel_matrix_numpy(points: np.ndarray, sigma: float, dtype=np.float64, block: int | None = None) -> np.ndarray:
    """X_ij = exp(-||x_i - x_j||^2 / sigma^2) with an exact unit diagonal (float64 math).

    With `block`, the matrix is built block by block (upper block triangle, mirrored), so that
    the peak memory is the result plus one block instead of several n x n temporaries."""
    if block is not None:
        return _kernel_matrix_blocked(points, sigma, dtype, block)
    sq = (points ** 2).sum(axis=1)
    d2 = sq[:, None] + sq[None, :] - 2.0 * (points @ points.T)
    np.maximum(d2, 0.0, out=d2)
    np.fill_diagonal(d2, 0.0)
    X = np.exp(-d2 / (sigma * sigma))
    X = 0.5 * (X + X.T)
    return X.astype(dtype, copy=False)


def _kernel_matrix_blocked(points, sigma, dtype, block):
    n = points.shape[0]
    sq = (points ** 2).sum(axis=1)
    X = np.empty((n, n), dtype=dtype)
    inv = 1.0 / (sigma * sigma)
    for r0 in range(0, n, block):
        r1 = min(n, r0 + block)
        for c0 in range(r0, n, block):
            c1 = min(n, c0 + block)
            d2 = sq[r0:r1, None] + sq[None, c0:c1] - 2.0 * (points[r0:r1] @ points[c0:c1].T)
            np.maximum(d2, 0.0, out=d2)
            if r0 == c0:
                np.fill_diagonal(d2, 0.0)
            blk = np.exp(-d2 * inv)
            if r0 == c0:
                blk = 0.5 * (blk + blk.T)
            X[r0:r1, c0:c1] = blk
            if c0 != r0:
                X[c0:c1, r0:r1] = blk.T
    return X


def kernel_matrix_torch(points, sigma: float, device, dtype=None, block: int = 4096, math_dtype=None):
    """Same kernel matrix built on a torch device, row block by row block.

    `points` is a numpy array; the result has `dtype` (default float32) and the
    distances are formed in `math_dtype` (default float64).  The matrix is
    symmetrised exactly by building only the upper block triangle and
    mirroring it.
    """
    import torch

    dtype = dtype or torch.float32
    P = torch.as_tensor(points, dtype=math_dtype or torch.float64, device=device)
    n = P.shape[0]
    sq = (P * P).sum(dim=1)
    X = torch.empty((n, n), dtype=dtype, device=device)
    inv = 1.0 / (sigma * sigma)
    for r0 in range(0, n, block):
        r1 = min(n, r0 + block)
        for c0 in range(r0, n, block):
            c1 = min(n, c0 + block)
            d2 = sq[r0:r1, None] + sq[None, c0:c1] - 2.0 * (P[r0:r1] @ P[c0:c1].T)
            d2.clamp_(min=0.0)
            if r0 == c0:
                d2.fill_diagonal_(0.0)
            blk = torch.exp(-d2 * inv)
            if r0 == c0:
                blk = 0.5 * (blk + blk.T)
            X[r0:r1, c0:c1] = blk.to(dtype)
            if c0 != r0:
                X[c0:c1, r0:r1] = blk.T.to(dtype)
    return X


# -------------------------------------------------------------- sparse SBM graph


def _unique_pairs(u: np.ndarray, v: np.ndarray):
    a = np.minimum(u, v).astype(np.int64)
    b = np.maximum(u, v).astype(np.int64)
    keep = a != b
    key = np.unique(a[keep] * (1 << 32) + b[keep])
    return (key >> 32), (key & 0xFFFFFFFF)


def sbm_csr(n: int = 1_000_000, c: int = 64, avg_deg: float = 30.0, ratio: float = 20.0,
            seed: int = 0, self_loops: bool = True, permute: bool = True):
    """Symmetric stochastic-block-model adjacency in CSR form.

    c equal communities of n_c = n / c nodes.  p_out solves
    (n_c - 1) p_in + (n - n_c) p_out = avg_deg with p_in = ratio * p_out.
    Edge counts per block pair are Binomial; endpoints are uniform within the
    blocks; duplicate pairs are merged.  Unit weights, X_ii = 1 when
    `self_loops`, node order shuffled by a fixed permutation when `permute`.

    Returns dict(row_ptr int64[n+1], col int32[nnz], val float32[nnz], labels int64[n]).
    """
    rng = np.random.default_rng(seed)
    nc = n // c
    sizes = np.full(c, nc)
    sizes[: n - nc * c] += 1
    starts = np.concatenate([[0], np.cumsum(sizes)])
    p_out = avg_deg / (ratio * (nc - 1) + (n - nc))
    p_in = ratio * p_out
    us, vs = [], []
    for b in range(c):
        s = int(sizes[b])
        m = rng.binomial(s * (s - 1) // 2, p_in)
        u = rng.integers(0, s, size=m) + starts[b]
        v = rng.integers(0, s, size=m) + starts[b]
        us.append(u)
        vs.append(v)
    pairs_out = (n * n - int((sizes.astype(np.int64) ** 2).sum())) // 2
    m = rng.binomial(pairs_out, p_out)
    labels_sorted = np.repeat(np.arange(c), sizes)
    got_u, got_v = [], []
    need = m
    while need > 0:
        u = rng.integers(0, n, size=int(need * 1.05) + 16)
        v = rng.integers(0, n, size=u.shape[0])
        ok = labels_sorted[u] != labels_sorted[v]
        u, v = u[ok][:need], v[ok][:need]
        got_u.append(u)
        got_v.append(v)
        need -= u.shape[0]
    us.extend(got_u)
    vs.extend(got_v)
    a, b = _unique_pairs(np.concatenate(us), np.concatenate(vs))
    perm = rng.permutation(n) if permute else np.arange(n)
    a = perm[a]
    b = perm[b]
    labels = np.empty(n, dtype=np.int64)
    labels[perm] = labels_sorted
    rows = np.concatenate([a, b])
    cols = np.concatenate([b, a])
    if self_loops:
        rows = np.concatenate([rows, np.arange(n)])
        cols = np.concatenate([cols, np.arange(n)])
    order = np.lexsort((cols, rows))
    rows = rows[order]
    cols = cols[order].astype(np.int32)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=row_ptr[1:])
    val = np.ones(cols.shape[0], dtype=np.float32)
    return dict(row_ptr=row_ptr, col=cols, val=val, labels=labels, n=n)


# ------------------------------------------------------------------ dense SBM


def dense_sbm(n: int, c: int, seed: int, p_in: float = 0.3, p_out: float = 0.015,
              dtype=np.float32):
    """Dense symmetric 0/1 SBM adjacency with a unit diagonal (communities shuffled)."""
    rng = np.random.default_rng(seed)
    labels = rng.permutation(np.arange(n) * c // n)
    P = np.where(labels[:, None] == labels[None, :], p_in, p_out)
    U = rng.random((n, n))
    A = np.triu(U < P, 1)
    A = A | A.T
    np.fill_diagonal(A, True)
    return A.astype(dtype), labels


def batched_problem_specs(nprob: int = 64, seed: int = 0, n_lo: int = 500, n_hi: int = 8000,
                          ks=(8, 12, 16, 24, 32)):
    """Sizes of the batched workload: n log-uniform in [n_lo, n_hi], k uniform over `ks`."""
    rng = np.random.default_rng(seed + 0xBA7C)
    ns = np.floor(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=nprob))).astype(int)
    kk = rng.choice(np.asarray(ks), size=nprob)
    return [dict(n=int(ns[p]), k=int(kk[p]), seed=int(p)) for p in range(nprob)]


def lvs_sample_count(k: int) -> int:
    """s = ceil(8 k ln k) rows per sampled update."""
    return int(math.ceil(8.0 * k * math.log(k)))
