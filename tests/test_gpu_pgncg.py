"""GPU parity of PGNCG-SymNMF and LAI-PGNCG-SymNMF with the FP64 oracle."""

import numpy as np
import pytest
import torch

from oracle import symnmf as O
from synth import gaussian_sketch, gmm_points, kernel_matrix_numpy, median_pair_distance, planted_dense, uniform_factor

from ._gpu_util import np64, rel_err, t32, t64

pytestmark = pytest.mark.gpu


def _gmm(n, seed):
    pts, _ = gmm_points(n, 10, 6, seed=seed)
    return kernel_matrix_numpy(pts, median_pair_distance(pts, seed=seed))


@pytest.mark.parametrize("s_max", [1, 5])
def test_pgncg_full_x_matches_oracle(S, s_max):
    n, k = 3000, 6
    X = _gmm(n, 41)
    H0 = (uniform_factor(n, k, seed=42) * O.init_scale(X, k)).astype(np.float32).astype(np.float64)
    s = S.Solver(t32(X), k, alpha=1.0)
    s.set_factors(t32(H0))
    got = s.pgncg(20, source=S.SRC_X, s_max=s_max)
    nx2 = float((X * X).sum())
    Href, ref = O.pgncg_symnmf(lambda F: X @ F, nx2, H0, 20, s_max=s_max)
    assert rel_err(got, ref).max() < 1e-4, rel_err(got, ref)
    Hg, Wg = s.factors()
    Hg = np64(Hg)
    np.testing.assert_array_equal(Hg, np64(Wg))  # W follows H
    np.testing.assert_allclose(Hg, Href, rtol=0, atol=1e-3 * np.abs(Href).max())


def test_lai_pgncg_matches_oracle_on_the_oracle_operator(S):
    n, k, l = 3000, 6, 22
    X = _gmm(n, 43)
    U, lam = O.apx_evd(X, gaussian_sketch(n, l, seed=44), 2)
    Uf = U.astype(np.float32).astype(np.float64)
    H0 = (uniform_factor(n, k, seed=45) * O.init_scale(X, k)).astype(np.float32).astype(np.float64)
    s = S.Solver(t32(X), k, alpha=1.0, max_width=l)
    s.set_lai(t32(U), lam)
    s.set_factors(t32(H0))
    got = s.pgncg(20, source=S.SRC_LAI, s_max=5)
    _, ref = O.pgncg_symnmf(lambda F: O.lai_product(Uf, lam, F), float((lam ** 2).sum()), H0, 20, s_max=5)
    assert rel_err(got, ref).max() < 1e-4, rel_err(got, ref)


def test_pgncg_on_bf16_x_and_gpu_sketch_reach_the_oracle_residual(S):
    # the mixed forms: BF16 X on the tensor cores, and LAI-PGNCG on the GPU's own sketch
    n, k, l = 4000, 8, 26
    X = _gmm(n, 46)
    H0 = (uniform_factor(n, k, seed=47) * O.init_scale(X, k)).astype(np.float32).astype(np.float64)
    nx2 = float((X * X).sum())
    Href, _ = O.pgncg_symnmf(lambda F: X @ F, nx2, H0, 25, s_max=5)
    nr_ref = O.symnmf_residual(X, Href)
    Xf = torch.tensor(X, dtype=torch.float32, device="cuda")
    sb = S.Solver(Xf.to(torch.bfloat16), k, alpha=1.0, x_hi=Xf, max_width=l)
    sb.set_factors(t32(H0))
    sb.pgncg(25, source=S.SRC_X, s_max=5, record=False)
    Hb = np64(sb.factors()[0])
    assert abs(O.symnmf_residual(X, Hb) - nr_ref) <= 1e-3
    sb.set_factors(t32(H0))
    sb.lai_sketch(l, 2)
    sb.pgncg(25, source=S.SRC_LAI, s_max=5, record=False)
    Hl = np64(sb.factors()[0])
    assert O.symnmf_residual(X, Hl) <= nr_ref + 1e-3


def test_pgncg_recovers_the_planted_factor(S):
    X, Hp, _ = planted_dense(n=1000, k=10, sigma=0.0, seed=1)
    rng = np.random.default_rng(5)
    s = S.Solver(t64(X), 10, alpha=1.0)
    s.set_factors(t32(Hp + 0.05 * rng.random(Hp.shape)))
    obj = s.pgncg(15, s_max=10)
    assert obj[-1] < obj[0]
    # the recovered factor, checked in FP64 on the host: ||X - H H^T|| / ||X|| at FP32 rounding
    assert O.symnmf_residual(X, np64(s.factors()[0])) < 1e-5
