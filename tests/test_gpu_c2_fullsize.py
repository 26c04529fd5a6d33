"""Full-size parity on the LAI benchmark instance (Alg. Apx-EVD, Alg. LAI-SymNMF).

Instance: n = 20000 points of a 20-component Gaussian mixture in R^50 (seed 0),
Gaussian kernel X, k = 20, l = 50, q = 2, Philox key 1, 200 sweeps, alpha = max(X).
The stored FP64 oracle trajectory is tests/golden/c2_reference.json (written by
tests/golden/make_c2_reference.py, which calls only oracle/ and synth/).
"""

import json
import os

import numpy as np
import pytest
import torch

from oracle import philox
from oracle import symnmf as O
from synth import gmm_points, kernel_matrix_numpy, kernel_matrix_torch, median_pair_distance

from ._gpu_util import np64, t32

pytestmark = pytest.mark.gpu

N, D, C, K, L, Q, SWEEPS, SEED = 20000, 50, 20, 20, 50, 2, 200, 1
MARKS = (1, 10, 50, 100, 200)
GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "c2_reference.json")))


@pytest.fixture(scope="module")
def points():
    pts, _ = gmm_points(N, D, C, seed=0)
    return pts, median_pair_distance(pts, seed=0)


@pytest.fixture(scope="module")
def xf(points):
    pts, sigma = points
    assert sigma == pytest.approx(GOLD["sigma"], rel=1e-15)
    return kernel_matrix_torch(pts, sigma, torch.device("cuda:0"))


def _solve(S, X, sweeps, **kw):
    s = S.Solver(X, K, max_width=L, seed=SEED, **kw)
    s.init_random(True)
    s.lai_sketch(L, Q)
    obj = s.sweep(sweeps, source=S.SRC_LAI)
    return s, obj


def test_fp32_sketch_and_200_lai_sweeps_match_stored_oracle(S, xf):
    # FP32 form end to end: GPU range finder + Apx-EVD on the FP32 X, then 200 LAI-HALS
    # sweeps in one persistent launch; objectives against the FP64 oracle at 1e-4 relative
    s, obj = _solve(S, xf, SWEEPS)
    alpha, _ = s.info()
    assert alpha == GOLD["alpha"]
    for t in MARKS:
        ref = GOLD["lai_obj"][str(t)]
        assert abs(obj[t - 1] - ref) <= 1e-4 * ref, (t, obj[t - 1], ref)
    # the true-X normalized residual of the final iterate (FP32 X, trace trick in FP64)
    nr, _ = s.residual(S.SRC_X)
    assert nr == pytest.approx(GOLD["lai_nr_true"], rel=1e-4)
    s.close()


@pytest.mark.parametrize("form", ["bf16", "fp8"])
def test_low_precision_forms_reach_the_oracle_residual(S, xf, form):
    # X stored BF16 / E4M3 with row scales for the sketch and the sweeps; the final true
    # residual (against the FP32 X) within 1e-3 absolute of the oracle's, two-sided
    if form == "bf16":
        s, _ = _solve(S, xf.to(torch.bfloat16), SWEEPS, x_hi=xf)
    else:
        x8, rs = S.quantize_fp8(xf)
        s, _ = _solve(S, x8, SWEEPS, row_scale=rs, x_hi=xf)
    nr, _ = s.residual(S.SRC_XHI)
    assert abs(nr - GOLD["lai_nr_true"]) <= 1e-3, (form, nr, GOLD["lai_nr_true"])
    s.close()


def test_engine_rows_match_oracle_on_the_oracle_operator(S, points, xf):
    # the persistent LAI sweep launch on the oracle's own U, Lambda (FP64 Apx-EVD of the FP64
    # X, U rounded to FP32 on both sides): W and H on 4096 sampled rows, element by element,
    # after 200 sweeps.  A float32 numpy restatement of these sweeps drifts 2.1e-5 (absolute,
    # max |H| = 0.91) from the FP64 oracle; the bound allows about five times that.
    pts, sigma = points
    X = kernel_matrix_numpy(pts, sigma)
    alpha = O.default_alpha(X)
    H0 = philox.philox_uniform_factor(N, K, SEED) * O.init_scale(X, K)
    U, lam = O.apx_evd(X, philox.philox_gaussian(N, L, SEED), Q)
    del X
    Uf = U.astype(np.float32).astype(np.float64)
    H0f = H0.astype(np.float32).astype(np.float64)
    W, H, ref = O.lai_symnmf(Uf, lam, H0f, alpha, SWEEPS)
    s = S.Solver(xf, K, max_width=L, alpha=alpha)
    s.set_lai(t32(U), lam)
    s.set_factors(t32(H0f))
    got = s.sweep(SWEEPS, source=S.SRC_LAI)
    dev = np.abs(np.asarray(got) - ref) / np.abs(ref)
    assert dev.max() < 1e-4, (dev.max(), int(dev.argmax()))
    Hg, Wg = s.factors()
    rows = np.random.default_rng(11).choice(N, 4096, replace=False)
    Hg, Wg = np64(Hg)[rows], np64(Wg)[rows]
    tol = 1e-4 * max(np.abs(H).max(), np.abs(W).max())
    np.testing.assert_allclose(Hg, H[rows], rtol=0, atol=tol)
    np.testing.assert_allclose(Wg, W[rows], rtol=0, atol=tol)
    s.close()
