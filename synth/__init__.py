"""Seeded synthetic inputs for the randomized SymNMF hot path.

This package generates the problem instances (data matrices X, initial factors,
Gaussian sketch matrices) that both the CUDA path and the CPU oracle consume.
It holds none of the method's arithmetic: no HALS, BPP, range finder,
leverage score or sampling step lives here, only the recipes that build the
inputs (planted block factors, Gaussian-mixture kernel matrices, stochastic
block model graphs).
"""

from .generators import (  # noqa: F401
    planted_dense,
    uniform_factor,
    gaussian_sketch,
    gmm_points,
    median_pair_distance,
    kernel_matrix_numpy,
    kernel_matrix_torch,
    sbm_csr,
    dense_sbm,
    batched_problem_specs,
    lvs_sample_count,
)
