"""GPU parity of LAI-SymNMF: range finder, Apx-EVD and the LAI sweeps."""

import numpy as np
import pytest
import torch

from oracle import symnmf as O
from synth import gaussian_sketch, gmm_points, kernel_matrix_numpy, median_pair_distance, planted_dense, uniform_factor

from ._gpu_util import np64, rel_err, t32, t64

pytestmark = pytest.mark.gpu


def _gmm_kernel(n, d, c, seed):
    pts, labels = gmm_points(n, d, c, seed=seed)
    return kernel_matrix_numpy(pts, median_pair_distance(pts, seed=seed)), labels


@pytest.mark.parametrize("lai_mode", [0, 1])  # one-launch CholeskyQR3, separate kernels per pass
def test_lai_operator_matches_oracle(S, lai_mode):
    X, _ = _gmm_kernel(2000, 10, 8, seed=0)
    l, q, k = 30, 2, 10
    Om = gaussian_sketch(2000, l, seed=1)
    s = S.Solver(t32(X), k, max_width=l, lai_mode=lai_mode)
    s.lai_sketch(l, q, t32(Om))
    U, lam = s.lai()
    Ug = np64(U)
    Uo, lo = O.apx_evd(X, Om, q)
    F = uniform_factor(2000, k, seed=2)
    got = Ug @ (lam[:, None] * (Ug.T @ F))
    ref = O.lai_product(Uo, lo, F)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-4
    np.testing.assert_allclose(Ug.T @ Ug, np.eye(l), atol=2e-5)
    np.testing.assert_allclose(np.sort(lam), np.sort(lo), rtol=1e-4, atol=1e-5 * np.abs(lo).max())


@pytest.mark.parametrize("lai_mode", [0, 1])
def test_exact_range_capture_rank_deficient(S, lai_mode):
    # planted X of rank 8 < l = 26: the rank-safe CholeskyQR3 keeps the captured range
    X, _, _ = planted_dense(n=800, k=8, sigma=0.0, seed=3)
    s = S.Solver(t64(X), 8, max_width=26, lai_mode=lai_mode)
    s.lai_sketch(26, 1)
    U, lam = s.lai()
    Ug = np64(U)
    A = Ug @ np.diag(lam) @ Ug.T
    assert np.linalg.norm(X - A) / np.linalg.norm(X) < 1e-5


@pytest.mark.parametrize("mode", ["engine", "graph", "eager"])
def test_lai_sweeps_match_oracle(S, mode):
    # sweeps on the oracle's own U, Lambda (given through symnmf_set_lai): parity of the
    # LAI-SymNMF loop itself, independent of the sketch's FP32 rounding
    X, _ = _gmm_kernel(3000, 10, 6, seed=4)
    k, l, q = 6, 22, 2
    U, lam = O.apx_evd(X, gaussian_sketch(3000, l, seed=5), q)
    Hi = uniform_factor(3000, k, seed=6) * O.init_scale(X, k)
    s = S.Solver(t32(X), k, max_width=l, use_graph=(mode == "graph"), lai_mode=(0 if mode == "engine" else 1))
    s.set_lai(t32(U), lam)
    s.set_factors(t32(Hi))
    got = s.sweep(100, source=S.SRC_LAI)
    Uf = U.astype(np.float32).astype(np.float64)
    _, _, ref = O.lai_symnmf(Uf, lam, Hi.astype(np.float32).astype(np.float64), O.default_alpha(X), 100)
    assert rel_err(got, ref).max() < 1e-4


def test_lai_sketch_then_sweeps_reach_oracle_residual(S):
    # end to end: GPU sketch (same Omega) + 100 LAI sweeps; final true residual vs the oracle's
    X, _ = _gmm_kernel(3000, 10, 6, seed=4)
    k, l, q = 6, 22, 2
    Om = gaussian_sketch(3000, l, seed=5)
    Hi = uniform_factor(3000, k, seed=6) * O.init_scale(X, k)
    s = S.Solver(t32(X), k, max_width=l)
    s.lai_sketch(l, q, t32(Om))
    s.set_factors(t32(Hi))
    s.sweep(100, source=S.SRC_LAI, record=False)
    nr, _ = s.residual(S.SRC_X)
    U, lam = O.apx_evd(X, Om, q)
    W, H, _ = O.lai_symnmf(U, lam, Hi, O.default_alpha(X), 100, record=False)
    assert abs(nr - O.normalized_residual(X, W, H)) <= 1e-4 * O.normalized_residual(X, W, H)


def test_lai_bf16_then_fp32_refinement_reaches_oracle_residual(S):
    # X stored BF16 for the sketch, FP32 copy for the refinement sweeps (Iterative Refinement)
    n, k, l, q = 4000, 8, 26, 2
    X, _ = _gmm_kernel(n, 12, 8, seed=7)
    Xf = torch.tensor(X, dtype=torch.float32, device="cuda")
    Xb = Xf.to(torch.bfloat16)
    Hi = uniform_factor(n, k, seed=8) * O.init_scale(X, k)
    alpha = O.default_alpha(X)
    W, H, _ = O.hals_symnmf(X, Hi, alpha, 60, record=False)
    nr_oracle = O.normalized_residual(X, W, H)
    s = S.Solver(Xb, k, x_hi=Xf, max_width=l)
    s.lai_sketch(l, q)
    s.set_factors(t32(Hi))
    s.sweep(60, source=S.SRC_LAI, record=False)
    s.sweep(5, source=S.SRC_XHI, record=False)
    nr, _ = s.residual(S.SRC_XHI)
    assert nr <= nr_oracle + 1e-3


def test_lai_fp8_sketch_is_close(S):
    n, k, l = 3000, 8, 26
    X, _ = _gmm_kernel(n, 12, 8, seed=9)
    Xf = torch.tensor(X, dtype=torch.float32, device="cuda")
    x8, rs = S.quantize_fp8(Xf)
    s = S.Solver(x8, k, row_scale=rs, x_hi=Xf, max_width=l)
    s.lai_sketch(l, 2)
    Hi = uniform_factor(n, k, seed=10) * O.init_scale(X, k)
    s.set_factors(t32(Hi))
    s.sweep(60, source=S.SRC_LAI, record=False)
    s.sweep(5, source=S.SRC_XHI, record=False)
    nr, _ = s.residual(S.SRC_XHI)
    W, H, _ = O.hals_symnmf(X, Hi, O.default_alpha(X), 60, record=False)
    assert nr <= O.normalized_residual(X, W, H) + 1e-3


@pytest.mark.parametrize("n,k,l", [(20000, 20, 50), (5003, 32, 74), (777, 64, 96), (50, 3, 8)])
def test_lai_engine_and_per_kernel_path_match_oracle(S, n, k, l):
    # both LAI sweep implementations on the oracle's U, Lambda of a rank-l operator
    rng = np.random.default_rng(n)
    Q, _ = np.linalg.qr(rng.standard_normal((n, l)))
    lam = np.sort(rng.uniform(0.1, 50.0, size=l))[::-1] * rng.choice([1, 1, 1, -1], size=l)
    Hi = rng.random((n, k)) * 0.1
    Uf = Q.astype(np.float32).astype(np.float64)
    alpha = 1.0
    _, Href, ref = O.lai_symnmf(Uf, lam, Hi.astype(np.float32).astype(np.float64), alpha, 30)
    Xdummy = torch.zeros((n, n), dtype=torch.float32, device="cuda")
    for mode in (0, 1, 2):  # resident engine, per-kernel path, streamed engine
        s = S.Solver(Xdummy, k, max_width=l, lai_mode=mode, alpha=alpha)
        s.set_lai(t32(Q), lam)
        s.set_factors(t32(Hi))
        got = s.sweep(30, source=S.SRC_LAI)
        assert rel_err(got, ref).max() < 1e-4, (mode, rel_err(got, ref).max())


@pytest.mark.parametrize("q_max", [0, 1, 8])
def test_ada_rrf_matches_oracle(S, q_max):
    # Alg. Ada-RRF on the GPU (FP32 X, same Omega): the same number of checks, residuals within
    # FP32 rounding of the oracle's, and the same LAI operator
    X, _ = _gmm_kernel(3000, 10, 6, seed=12)
    l = 22
    Om = gaussian_sketch(3000, l, seed=13)
    s = S.Solver(t32(X), 6, max_width=l)
    got = s.lai_sketch_ada(l, q_max, 1e-3, t32(Om))
    Uo, lo, hist, passes = O.apx_evd_ada(X, Om, q_max, 1e-3)
    assert got["checks"] == len(hist) and got["passes"] == passes
    np.testing.assert_allclose(got["nr_hist"], hist, rtol=0, atol=2e-5)
    U, lam = s.lai()
    Ug = np64(U)
    F = uniform_factor(3000, 6, seed=14)
    ref = O.lai_product(Uo, lo, F)
    assert np.linalg.norm(Ug @ (lam[:, None] * (Ug.T @ F)) - ref) / np.linalg.norm(ref) < 1e-4


def test_ada_rrf_stops_early_on_a_low_rank_matrix(S):
    X, _, _ = planted_dense(n=800, k=8, sigma=0.0, seed=3)
    s = S.Solver(t64(X), 8, max_width=26)
    got = s.lai_sketch_ada(26, 10, 1e-3)
    assert got["checks"] == 2 and got["passes"] == 5
    # sqrt(||X||^2 - ||B||^2) / ||X|| from FP32 products cancels down to ~sqrt(FP32 eps)
    assert got["nr_hist"][0] < 1e-3
    U, lam = s.lai()
    Ug = np64(U)
    assert np.linalg.norm(X - (Ug * lam) @ Ug.T) / np.linalg.norm(X) < 1e-5


@pytest.mark.parametrize("rule", ["hals", "bpp"])
def test_compressed_sweeps_match_oracle(S, rule):
    # Compressed-SymNMF on the GPU's sketch basis (same Omega) against the oracle's on its
    # Householder basis: the compressed problem depends only on the projector Q Q^T
    X, _ = _gmm_kernel(3000, 10, 6, seed=15)
    k, l, q = 6, 22, 2
    Om = gaussian_sketch(3000, l, seed=16)
    Hi = (uniform_factor(3000, k, seed=17) * O.init_scale(X, k)).astype(np.float32).astype(np.float64)
    r = S.RULE_HALS if rule == "hals" else S.RULE_BPP
    s = S.Solver(t32(X), k, max_width=l)
    s.lai_sketch(l, q, t32(Om))
    s.set_factors(t32(Hi))
    got = s.sweep(30, source=S.SRC_COMP, rule=r)
    Q = O.rrf(X, Om, q)
    W, H, ref = O.compressed_symnmf(X, Q, Hi, O.default_alpha(X), 30, rule=rule)
    assert rel_err(got, ref).max() < 1e-4, rel_err(got, ref).max()
    Hg, Wg = s.factors()
    np.testing.assert_allclose(np64(Hg), H, rtol=0, atol=1e-3 * np.abs(H).max())
    # not a residual source
    with pytest.raises(S.SymNMFError):
        s.residual(S.SRC_COMP)


def test_paper_schedule_matches_oracle(S):
    # the experiments' schedule: Ada-RRF (1e-3), LAI-HALS to the 1e-4 x 4 stopping rule, then
    # Iterative Refinement on X with the same rule, against the oracle's run of the same schedule
    from oracle import philox

    X, _ = _gmm_kernel(2000, 10, 6, seed=18)
    n, k, l, seed = 2000, 6, 22, 9
    Hi = (uniform_factor(n, k, seed=19) * O.init_scale(X, k)).astype(np.float32).astype(np.float64)
    s = S.Solver(t32(X), k, max_width=l, seed=seed)
    s.set_factors(t32(Hi))
    got = s.solve(method=S.SRC_LAI, l=l, q_max=8, max_iters=300, max_refine=300)
    ref = O.lai_schedule(X, philox.philox_gaussian(n, l, seed), Hi, O.default_alpha(X), q_max=8, max_iters=300,
                         max_refine=300)
    assert got["checks"] == ref["checks"] and got["passes"] == ref["passes"]
    assert abs(got["iters"] - ref["iters"]) <= 2, (got, ref["iters"])
    assert abs(got["refine_iters"] - ref["refine_iters"]) <= 3, (got, ref["refine_iters"])
    assert abs(got["nr_final"] - ref["nr_final"]) <= 2e-4
    # the full-X and compressed methods run through the same driver
    s.set_factors(t32(Hi))
    full = s.solve(method=S.SRC_X, max_iters=300)
    assert full["iters"] < 300 and full["checks"] == 0
    s.set_factors(t32(Hi))
    comp = s.solve(method=S.SRC_COMP, l=l, q_max=8, max_iters=300, max_refine=300)
    assert comp["nr_final"] <= full["nr_final"] + 1e-2


@pytest.mark.parametrize("xfmt", ["bf16", "f32"])
def test_sweep_to_target_stops_where_host_checks_stop(S, xfmt):
    # symnmf_sweep_to_target decides on the device (LAI engine: one graph with a WHILE node); it must
    # stop at the same check, with the same residual and factors, as sweeps and checks issued one by
    # one from the host (same kernels in the same order: equal to the last bit)
    n, k, l, q = 3000, 6, 22, 2
    X, _ = _gmm_kernel(n, 10, 6, seed=4)
    Xt = t32(X) if xfmt == "f32" else t32(X).to(torch.bfloat16)
    Om = gaussian_sketch(n, l, seed=5)
    Hi = uniform_factor(n, k, seed=6) * O.init_scale(X, k)

    def fresh():
        s = S.Solver(Xt, k, max_width=l)
        s.lai_sketch(l, q, t32(Om))
        s.set_factors(t32(Hi))
        return s

    a = fresh()
    nrs = []
    for _ in range(14):
        a.sweep(10, source=S.SRC_LAI, record=False)
        nrs.append(a.residual(S.SRC_X)[0])
    assert all(np.isfinite(nrs))
    # the first check at or below the target is check 7 (index 6)
    stop = 6
    target = nrs[stop]
    assert min(nrs[:stop]) > target
    b = fresh()
    r = b.sweep_to_target(target, chunk=10, max_sweeps=200)
    assert (r["checks"], r["sweeps"]) == (stop + 1, 10 * (stop + 1))
    assert r["nr"] == nrs[stop]
    c = fresh()
    for _ in range(stop + 1):
        c.sweep(10, source=S.SRC_LAI, record=False)
    for got, ref in zip(b.factors(), c.factors()):
        assert torch.equal(got, ref)
    # a target never reached: every allowed check, the last one's residual
    d = fresh()
    r = d.sweep_to_target(0.0, chunk=10, max_sweeps=50)
    assert (r["checks"], r["sweeps"], r["nr"]) == (5, 50, nrs[4])
    # reached at the first check (no graph launch)
    e = fresh()
    r = e.sweep_to_target(1.0, chunk=10, max_sweeps=200)
    assert (r["checks"], r["sweeps"], r["nr"]) == (1, 10, nrs[0])
    # the same solve again on the same handle: the repeated call records the device loop (one graph
    # with a WHILE node), the third replays it
    for rep in range(2):
        b.set_factors(t32(Hi))
        r = b.sweep_to_target(target, chunk=10, max_sweeps=200)
        assert (r["checks"], r["sweeps"], r["nr"]) == (stop + 1, 10 * (stop + 1), nrs[stop]), rep
        for got, ref in zip(b.factors(), c.factors()):
            assert torch.equal(got, ref)
    # a device loop that continues from the previous call's state and uses all its checks
    b.sweep_to_target(0.0, chunk=10, max_sweeps=30)
    r = b.sweep_to_target(0.0, chunk=10, max_sweeps=30)
    assert (r["checks"], r["sweeps"], r["nr"]) == (3, 30, nrs[stop + 6])


def test_sweep_to_target_host_checked_sources(S):
    # full-X sweeps are checked on the host after each chunk; a ragged last chunk is cut to max_sweeps
    n, k = 2000, 5
    X, _ = _gmm_kernel(n, 8, 5, seed=9)
    Hi = uniform_factor(n, k, seed=10) * O.init_scale(X, k)
    a = S.Solver(t32(X), k)
    a.set_factors(t32(Hi))
    nrs = []
    for m in (7, 7, 6):
        a.sweep(m, source=S.SRC_X, record=False)
        nrs.append(a.residual(S.SRC_X)[0])
    b = S.Solver(t32(X), k)
    b.set_factors(t32(Hi))
    r = b.sweep_to_target(0.0, source=S.SRC_X, check=S.SRC_X, chunk=7, max_sweeps=20)
    assert (r["checks"], r["sweeps"], r["nr"]) == (3, 20, nrs[2])
    with pytest.raises(S.SymNMFError):
        b.sweep_to_target(0.0, source=S.SRC_LAI, chunk=10, max_sweeps=20)  # no sketch yet
