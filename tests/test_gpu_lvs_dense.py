"""LvS-SymNMF on dense X and LvS-BPP at the paper's sparse-graph settings (Alg. LvS-SymNMF).

The paper's sparse runs use k = 16, s = ceil(0.05 m), tau = 1/s with the HALS and BPP
update rules; it could not run the dense case in MATLAB (copying sampled rows of a
large dense X each iteration).  On the GPU the sampled columns of a dense symmetric X
are its sampled rows, read contiguously.

Each half step is checked against the FP64 oracle from the GPU's current factors: the
oracle's leverage scores of the GPU's fixed factor are fed to the sampler (indices then
bit-exact), and the GPU's update must equal the oracle's Update on the same sample.
"""

import math

import numpy as np
import pytest
import scipy.sparse as sp
import torch

from oracle import symnmf as O
from synth import gmm_points, kernel_matrix_numpy, median_pair_distance, sbm_csr, uniform_factor

from ._gpu_util import np64, t32

pytestmark = pytest.mark.gpu

K = 16


def _dense(n, fmt):
    pts, _ = gmm_points(n, 10, 16, seed=31)
    X = kernel_matrix_numpy(pts, median_pair_distance(pts, seed=31))
    Xf = torch.tensor(X, dtype=torch.float32, device="cuda")
    if fmt == "bf16":
        Xd = Xf.to(torch.bfloat16)
        return Xd, np64(Xd)
    return Xf, np64(Xf)


def _stepwise(S, s, Xo, n, rule, iters, seed, alpha):
    ns = math.ceil(0.05 * n)
    tau = 1.0 / ns
    for it in range(iters):
        for side in (0, 1):
            H, W = s.factors()
            H, W = np64(H), np64(W)
            Ffix, Fold = (H, W) if side == 0 else (W, H)
            # a column that HALS zeroed makes F^T F singular: the oracle's pseudo-inverse scores
            # (the paper's rank-deficient reading) are fed to the sampler all the same
            lev, _ = O.leverage_scores(Ffix)
            got = s.lvs_sample(side, it, tau, ns, lev_in=lev)
            ref = O.hybrid_sample(lev, K, ns, tau, seed=seed, it=it, side=side)
            np.testing.assert_array_equal(got["idx"], ref["idx"])
            assert got["s_D"] == ref["s_D"]
            s.lvs_update(side, rule)
            Y, G = O.sampled_products(Xo, Ffix, ref["idx"], ref["wt"])
            if rule == S.RULE_HALS:
                new_ref = O.hals_update_efficient(Fold, Ffix, G, Y, alpha)
            else:
                new_ref = O.bpp_update(Ffix, G, Y, alpha)
            Hn, Wn = s.factors()
            new = np64(Wn if side == 0 else Hn)
            scale = np.abs(new_ref).max()
            np.testing.assert_allclose(new, new_ref, rtol=0, atol=2e-4 * scale,
                                       err_msg=f"iteration {it} side {side}")


@pytest.mark.parametrize("fmt", ["f32", "bf16"])
@pytest.mark.parametrize("rule", ["hals", "bpp"])
def test_dense_lvs_half_steps_match_oracle(S, fmt, rule):
    n = 4000
    Xd, Xo = _dense(n, fmt)
    alpha = float(Xo.max())
    s = S.Solver(Xd, K, seed=101, alpha=alpha)
    s.set_factors(t32(uniform_factor(n, K, seed=5) * O.init_scale(Xo, K)))
    _stepwise(S, s, Xo, n, S.RULE_HALS if rule == "hals" else S.RULE_BPP, 4, 101, alpha)


@pytest.mark.parametrize("rule", ["hals", "bpp"])
def test_sparse_lvs_bpp_and_hals_at_paper_settings(S, rule):
    # stochastic block model (unit weights, self loops), k = 16, s = ceil(0.05 m), tau = 1/s
    n = 20000
    g = sbm_csr(n=n, c=16, avg_deg=30.0, ratio=20, seed=9)
    Xo = sp.csr_matrix((g["val"].astype(np.float64), g["col"], g["row_ptr"]), shape=(n, n))
    dev = [torch.tensor(g[a], device="cuda") for a in ("row_ptr", "col", "val")]
    s = S.Solver(csr=tuple(dev), k=K, n=n, seed=202)
    s.set_factors(t32(uniform_factor(n, K, seed=6)))
    _stepwise(S, s, Xo, n, S.RULE_HALS if rule == "hals" else S.RULE_BPP, 3, 202, 1.0)


@pytest.mark.parametrize("rule", ["hals", "bpp"])
def test_dense_lvs_iterations_reduce_the_residual(S, rule):
    # whole LvS iterations on the device (GPU leverage scores): the residual falls from the start and
    # ends near the full-X solver's after the same number of iterations (sampling costs a little)
    n = 4000
    Xd, Xo = _dense(n, "f32")
    alpha = float(Xo.max())
    H0 = t32(uniform_factor(n, K, seed=8) * O.init_scale(Xo, K))
    s = S.Solver(Xd, K, seed=303, alpha=alpha)
    s.set_factors(H0)
    nr0 = s.residual(S.SRC_X)[0]
    r = S.RULE_HALS if rule == "hals" else S.RULE_BPP
    s.lvs_iterate(30, 1.0 / math.ceil(0.05 * n), math.ceil(0.05 * n), rule=r)
    nr_lvs = s.residual(S.SRC_X)[0]
    f = S.Solver(Xd, K, seed=303, alpha=alpha)
    f.set_factors(H0)
    f.sweep(30, rule=r, record=False)
    nr_full = f.residual(S.SRC_X)[0]
    assert nr_lvs < 0.5 * nr0
    assert nr_lvs <= nr_full + 0.02, (nr_lvs, nr_full)
