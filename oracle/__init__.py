"""FP64 CPU oracle for randomized SymNMF (Hayashi, Aksoy, Ballard, Park; arXiv 2402.08134).

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
benchmark's CPU-baseline / reference leg may import this package.  The
library under `paper_2402_08134_gb300/` never imports it and shares no code
with it: the CUDA path and this oracle are independent restatements of the
paper, compared element by element in the tests.

Everything is plain numpy/scipy in float64, written step by step in the
paper's order and notation:

* `philox`  - Philox4x32-10 counter generator (Salmon et al., SC'11) and the
  Box-Muller / uniform streams built on it;
* `symnmf`  - regularised HALS (Eq. symhals_update1/2), standard HALS, the
  ANLS/BPP row solves, RRF + Apx-EVD, LAI-SymNMF, leverage scores via
  CholeskyQR, hybrid leverage-score sampling, LvS-SymNMF, residuals and
  projected gradients;
* `mlp`     - forward/backward of the 3-layer warm-start network and its
  Gram-matching loss.

Pins: every function is checked in `tests/test_oracle_*.py` against
something other than itself (closed forms, LAPACK, brute force, finite
differences, published known-answer vectors).  Functions with no such pin
say "parity unpinned" in their docstring.
"""
