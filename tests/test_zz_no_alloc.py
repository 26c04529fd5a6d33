"""The allocation-free Gram entry point (for callers that must not allocate device memory).

Collected last on purpose (file name), so that a run stopping at the first failure
has already run every other test.  It must also pass alone in a fresh process.
"""

import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _gram_via_abi(S, fn, F):
    n, N = F.shape
    G = torch.empty((N, N), dtype=torch.float64, device=F.device)
    st = fn(C.c_void_p(F.data_ptr()), n, N, C.c_void_p(G.data_ptr()),
            C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == S.OK, S.STATUS_NAMES.get(st, st)
    torch.cuda.synchronize()
    return G.cpu().numpy()


@pytest.mark.parametrize("n,N", [(20000, 20), (100003, 64), (5, 3)])
def test_gram_noalloc_matches_allocating_gram_twice(S, n, N):
    g = torch.Generator(device="cuda").manual_seed(n + N)
    for call in range(2):  # the static scratch keeps the last call's contents
        F = torch.rand((n, N), device="cuda", generator=g)
        ref = _gram_via_abi(S, S.symnmf_gram, F)
        got = _gram_via_abi(S, S.symnmf_gram_noalloc, F)
        exact = F.double().T @ F.double()
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(got, exact.cpu().numpy(), rtol=2e-7, atol=1e-12)


def test_gram_noalloc_rejects_wide_factors(S):
    F = torch.rand((100, 65), device="cuda")
    G = torch.empty((65, 65), dtype=torch.float64, device="cuda")
    st = S.symnmf_gram_noalloc(C.c_void_p(F.data_ptr()), 100, 65, C.c_void_p(G.data_ptr()), None)
    assert st == S.EINVAL
