"""GPU parity of the standalone kernels against the oracle / exact references."""

import numpy as np
import pytest
import scipy.sparse as sp
import torch

from oracle import philox
from synth import gmm_points, kernel_matrix_numpy, median_pair_distance, sbm_csr, uniform_factor

from ._gpu_util import np64, product_bound, t32, t64

pytestmark = pytest.mark.gpu


def _fp8_col_scale(Ft):
    """Column scales of the E4M3 packing: max |F[:, c]| / 448 by IEEE division in float32 (1 for a
    zero column).  torch's division by a Python scalar multiplies by a rounded reciprocal instead,
    which can move a scale by one ulp and, through it, flip an E4M3 rounding of that column."""
    mx = Ft.abs().amax(dim=0).cpu().numpy().astype(np.float32)
    cs = np.where(mx > 0, mx / np.float32(448.0), np.float32(1.0)).astype(np.float32)
    return torch.tensor(cs, device=Ft.device)


def _sym(n, seed):
    rng = np.random.default_rng(seed)
    A = rng.random((n, n))
    return 0.5 * (A + A.T)


def test_philox_gaussian_matches_oracle(S):
    for n, l, seed in [(1000, 50, 7), (333, 17, 2**40 + 5)]:
        got = np64(S.gaussian(n, l, seed))
        ref = philox.philox_gaussian(n, l, seed).astype(np.float32).astype(np.float64)
        np.testing.assert_allclose(got, ref, rtol=3e-7, atol=3e-7)


@pytest.mark.parametrize("n", [1000, 1157])
@pytest.mark.parametrize("N", [10, 20, 50, 100])
def test_simt_product_f32_and_f64(S, n, N):
    X = _sym(n, n + N)
    F = uniform_factor(n, N, seed=N)
    ref = X @ F
    Y32 = np64(S.dense_xf(t32(X), t32(F), gemm=S.GEMM_SIMT))
    assert (np.abs(Y32 - ref) <= product_bound(X, F, 2e-6)).all()
    Y64 = np64(S.dense_xf(t64(X), t32(F), gemm=S.GEMM_SIMT))
    F32 = F.astype(np.float32).astype(np.float64)
    np.testing.assert_allclose(Y64, X @ F32, rtol=1e-6)


@pytest.mark.parametrize("n", [1000, 4104, 20000])
@pytest.mark.parametrize("N", [10, 20, 50, 64, 100, 200, 256, 300, 512])  # 256: 256-row tiles; 512: wide
def test_tcgen05_bf16_product(S, n, N):
    if n == 20000 and N not in (20, 50):
        pytest.skip("full size only at the sketch widths")
    rng = np.random.default_rng(n * 7 + N)
    X = rng.random((n, n), dtype=np.float32)
    Xb = torch.tensor(X, device="cuda").to(torch.bfloat16)
    ld = (n + 7) // 8 * 8
    if ld != n:
        pad = torch.zeros((n, ld), dtype=torch.bfloat16, device="cuda")
        pad[:, :n] = Xb
        Xb = pad
    F = rng.standard_normal((n, N)).astype(np.float32)
    Fb = torch.tensor(F, device="cuda").to(torch.bfloat16).double().cpu().numpy()
    Xe = Xb[:, :n].double().cpu().numpy()
    Y = np64(S.dense_xf(Xb[:, :n] if ld == n else Xb, t32(F), gemm=S.GEMM_TC, N=N))
    ref = Xe @ Fb
    bound = product_bound(Xe, Fb, 2e-6)
    assert (np.abs(Y - ref) <= bound).all(), np.abs(Y - ref).max()


@pytest.mark.parametrize("fmt", ["bf16", "fp8"])
@pytest.mark.parametrize("N", [20, 50, 128])
def test_tcgen05_product_is_unbiased_over_long_k(S, fmt, N):
    # nonnegative X and F (as in SymNMF): the mean signed relative error of Y against the exact
    # product of the rounded operands must (nearly) vanish.  Tensor-core accumulation drifts low
    # by ~2e-8 relative per MMA; over K = 20000 in one accumulator that was 6e-5, which the
    # trace-trick residual (a difference of terms ~ ||X||^2) turns into a 4e-3 error in NR.  With
    # accumulations of 8 k blocks (32 MMAs) added in FP32 registers it is ~7e-7 (NR: ~4e-5).
    n = 20000
    rng = np.random.default_rng(N + (fmt == "fp8"))
    Xt = torch.rand((n, n), device="cuda", generator=torch.Generator(device="cuda").manual_seed(N))
    F = rng.random((n, N)).astype(np.float32)
    Ft = t32(F)
    if fmt == "bf16":
        Xq = Xt.to(torch.bfloat16)
        Y = S.dense_xf(Xq, Ft, gemm=S.GEMM_TC)
        ref = Xq.double() @ Ft.to(torch.bfloat16).double()
    else:
        x8, rs = S.quantize_fp8(Xt)
        Y = S.dense_xf(x8, Ft, row_scale=rs, gemm=S.GEMM_TC)
        Xe = x8[:, :n].view(torch.float8_e4m3fn).double() * rs.double()[:, None]
        cs = _fp8_col_scale(Ft)
        Fq = (Ft / cs).to(torch.float8_e4m3fn).double() * cs.double()
        ref = Xe @ Fq
    rel = ((Y.double() - ref) / ref).cpu().numpy()
    assert abs(rel.mean()) < 1.5e-6, rel.mean()
    assert np.abs(rel).max() < 1e-4


@pytest.mark.parametrize("n,N", [(1000, 20), (2064, 50), (4096, 128), (3000, 256), (333, 160), (2048, 512),
                                 (777, 400)])
def test_tcgen05_fp8_product(S, n, N):
    rng = np.random.default_rng(n + N)
    X = _sym(n, n).astype(np.float32)
    Xt = torch.tensor(X, device="cuda")
    x8, rs = S.quantize_fp8(Xt)
    F = rng.random((n, N)).astype(np.float32)
    Y = np64(S.dense_xf(x8[:, :n] if x8.shape[1] == n else x8, t32(F), row_scale=rs, gemm=S.GEMM_TC, N=N))
    # reference: the same E4M3 codes, dequantised, times the E4M3-quantised F
    Xq = x8[:, :n].view(torch.float8_e4m3fn).double() * rs.double()[:, None]
    Ft = t32(F)
    cs = _fp8_col_scale(Ft)
    Fq = (Ft / cs).to(torch.float8_e4m3fn).double() * cs.double()
    ref = (Xq @ Fq).cpu().numpy()
    bound = product_bound(Xq.cpu().numpy(), Fq.cpu().numpy(), 2e-6)
    assert (np.abs(Y - ref) <= bound).all(), np.abs(Y - ref).max()
    # and the quantised product stays close to the exact one (E4M3 steps)
    exact = X.astype(np.float64) @ F.astype(np.float64)
    assert np.abs(Y - exact).max() / np.abs(exact).max() < 0.05


def test_fp8_quantizer_and_bf16_convert(S):
    n = 777
    X = _sym(n, 3).astype(np.float32)
    X[5] = 0.0
    X[:, 5] = 0.0
    Xt = torch.tensor(X, device="cuda")
    x8, rs = S.quantize_fp8(Xt)
    mx = np.abs(X).max(axis=1)
    ref_rs = np.where(mx > 0, mx / 448.0, 1.0).astype(np.float32)
    np.testing.assert_allclose(rs.cpu().numpy(), ref_rs, rtol=1e-7)
    ref8 = (Xt / rs[:, None]).to(torch.float8_e4m3fn).view(torch.uint8)
    assert torch.equal(x8[:, :n], ref8)
    assert int(x8[:, n:].abs().sum()) == 0
    xb = S.convert_bf16(Xt)
    assert torch.equal(xb[:, :n], Xt.to(torch.bfloat16))


def test_csr_product(S):
    g = sbm_csr(n=5000, c=8, avg_deg=20, ratio=10, seed=1)
    Xs = sp.csr_matrix((g["val"].astype(np.float64), g["col"], g["row_ptr"]), shape=(5000, 5000))
    for N in (3, 16, 20, 50, 64, 74, 128):  # <= 16: half a warp per row; 50, 74: rows not aligned for vector loads
        F = uniform_factor(5000, N, seed=N)
        rp = torch.tensor(g["row_ptr"], device="cuda")
        col = torch.tensor(g["col"], device="cuda")
        val = torch.tensor(g["val"], device="cuda")
        Y = np64(S.csr_xf(rp, col, val, t32(F)))
        ref = Xs @ F.astype(np.float32).astype(np.float64)
        np.testing.assert_allclose(Y, ref, rtol=2e-6, atol=1e-6)


@pytest.mark.parametrize("n,N", [(270001, 64), (1100003, 20), (2500003, 10), (4000001, 5)])
def test_csr_product_with_f_larger_than_l2(S, n, N):
    # F of 64 to 95 MB: the gathers of F rows miss L2; every width path (N = 5, 10: half a warp
    # per row, 20: a warp, 64: float2 loads) against the exact product of the FP32 operands
    rng = np.random.default_rng(n)
    deg = 6
    rows = np.repeat(np.arange(n), deg)
    cols = rng.integers(0, n, size=n * deg)
    Xs = sp.csr_matrix((rng.random(n * deg), (rows, cols)), shape=(n, n))
    Xs.sum_duplicates()
    Xs.sort_indices()
    F = rng.random((n, N)).astype(np.float32)
    rp = torch.tensor(Xs.indptr.astype(np.int64), device="cuda")
    col = torch.tensor(Xs.indices.astype(np.int32), device="cuda")
    val = torch.tensor(Xs.data.astype(np.float32), device="cuda")
    Y = np64(S.csr_xf(rp, col, val, t32(F)))
    Xe = sp.csr_matrix((Xs.data.astype(np.float32).astype(np.float64), Xs.indices, Xs.indptr), shape=(n, n))
    ref = Xe @ F.astype(np.float64)
    bound = 2e-6 * (abs(Xe) @ np.abs(F.astype(np.float64))) + 1e-30
    assert (np.abs(Y - ref) <= bound).all(), np.abs(Y - ref).max()


@pytest.mark.parametrize("n,N", [(1, 3), (50, 10), (20000, 64), (100003, 20), (3000, 96)])
def test_gram_fp64_accumulation(S, n, N):
    F = uniform_factor(n, N, seed=n).astype(np.float32).astype(np.float64)
    G = np64(S.gram(t32(F)))
    np.testing.assert_allclose(G, F.T @ F, rtol=2e-7, atol=1e-12)


def test_kernel_matrix_product_at_sketch_width(S):
    pts, _ = gmm_points(3000, 10, 5, seed=0)
    X = kernel_matrix_numpy(pts, median_pair_distance(pts, seed=0))
    Om = philox.philox_gaussian(3000, 30, 5)
    Y = np64(S.dense_xf(t32(X), t32(Om), gemm=S.GEMM_SIMT))
    assert (np.abs(Y - X @ Om) <= product_bound(X, Om, 3e-6)).all()
