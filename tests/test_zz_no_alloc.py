"""The allocation-free Gram entry point (for callers that must not allocate device memory).

Some callers cannot call cudaMalloc: code running inside a host application that owns
every byte of device memory through its own fixed pool, or a real-time loop where an
allocation (and the implicit synchronisation of cudaFree) is forbidden.
symnmf_gram_noalloc serves them with a static device scratch array instead.

Collected last on purpose (file name), so that a run stopping at the first failure
has already run every other test.  It must also pass alone in a fresh process.
"""

import ctypes as C
import ctypes.util
import os

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
        # both entry points run the same kernel with the same grid: same summation order
        np.testing.assert_array_equal(got, ref)
        np.testing.assert_allclose(got, exact.cpu().numpy(), rtol=2e-7, atol=1e-12)


def test_gram_noalloc_rejects_wide_factors(S):
    F = torch.rand((100, 65), device="cuda")
    G = torch.empty((65, 65), dtype=torch.float64, device="cuda")
    st = S.symnmf_gram_noalloc(C.c_void_p(F.data_ptr()), 100, 65, C.c_void_p(G.data_ptr()), None)
    assert st == S.EINVAL


def _cudart():
    """The toolkit's CUDA runtime, to read the device's default memory pool."""
    names = [ctypes.util.find_library("cudart"), "libcudart.so", "libcudart.so.13",
             "/usr/local/cuda/lib64/libcudart.so", "/usr/local/cuda/lib64/libcudart.so.13"]
    for nm in names:
        if not nm:
            continue
        try:
            return C.CDLL(nm)
        except OSError:
            continue
    return None


def test_gram_noalloc_leaves_default_pool_untouched(S):
    # symnmf_gram takes its scratch from the device's default stream-ordered pool; the
    # allocation-free entry point must not raise that pool's high-water mark
    rt = _cudart()
    if rt is None or not os.path.exists("/usr/local/cuda"):
        pytest.skip("CUDA runtime library not found")
    USED_CUR, USED_HIGH = 7, 8  # cudaMemPoolAttrUsedMemCurrent, cudaMemPoolAttrUsedMemHigh
    pool = C.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(C.byref(pool), torch.cuda.current_device()) == 0

    def read(attr):
        v = C.c_uint64()
        assert rt.cudaMemPoolGetAttribute(pool, attr, C.byref(v)) == 0
        return v.value

    def reset_high():
        z = C.c_uint64(0)
        assert rt.cudaMemPoolSetAttribute(pool, USED_HIGH, C.byref(z)) == 0

    F = torch.rand((50000, 64), device="cuda")
    torch.cuda.synchronize()
    grows = {}
    for name in ("symnmf_gram", "symnmf_gram_noalloc"):
        reset_high()
        base = read(USED_CUR)
        _gram_via_abi(S, getattr(S, name), F)
        grows[name] = read(USED_HIGH) - base
    assert grows["symnmf_gram"] > 0  # the check sees the allocating entry point's scratch
    assert grows["symnmf_gram_noalloc"] == 0
