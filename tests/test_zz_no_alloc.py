"""The allocation-free k-means++ entry point (raftgp_kmeanspp_noalloc) against the
workspace entry point (raftgp_kmeanspp), through the C ABI.

raftgp_kmeanspp_noalloc exists for callers that cannot allocate device memory (a plugin in
another program's CUDA context whose allocator owns the device memory, or a process that
reserves all its device memory up front); it keeps its scratch in a static device array.
Seeds are integers, so the two entry points must agree exactly; two calls in a row check
that the shared array's leftover contents from one call do not leak into the next.  A call
after the first must not change the device's free memory or torch's reserved pool, and the
largest accepted n must work.  This file runs last (pytest collects it after the others) and
also passes alone in a fresh process."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2312_01560_gb300 import _abi, api

pytestmark = pytest.mark.gpu

MAX_N = 4_500_000          # RAFTGP_NOALLOC_MAX_N


def _call(Z, K, seed, seeds):
    n, d = Z.shape
    code = 1 if Z.dtype == torch.bfloat16 else 0
    return _abi.lib().raftgp_kmeanspp_noalloc(C.c_void_p(Z.data_ptr()), n, d, code, K, seed,
                                              C.c_void_p(seeds.data_ptr()),
                                              C.c_void_p(torch.cuda.current_stream().cuda_stream))


def _noalloc(Z, K, seed):
    seeds = torch.full((K,), -1, dtype=torch.int32, device=Z.device)
    _abi.check(_call(Z, K, seed, seeds))
    torch.cuda.synchronize()
    return seeds


def _unit_rows(n, d, seed, dtype):
    rng = np.random.default_rng(seed)
    z = rng.normal(size=(n, d))
    z /= np.linalg.norm(z, axis=1, keepdims=True)
    return torch.tensor(z, dtype=dtype, device="cuda")


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_noalloc_matches_workspace_entry_point_twice(cuda, dtype):
    Z = _unit_rows(20011, 64, 1, dtype)
    calls = [(Z, 57, 5), (_unit_rows(3001, 32, 2, dtype), 400, 9)]   # second call: other shape, K, seed
    for Zc, K, seed in calls:
        ref = api.kmeanspp(Zc, K, seed).cpu().numpy()
        got = _noalloc(Zc, K, seed).cpu().numpy()
        assert np.array_equal(got, ref)
        assert len(set(got.tolist())) == K


def test_noalloc_call_allocates_no_device_memory(cuda):
    Z = _unit_rows(50000, 64, 4, torch.float32)
    seeds = torch.full((100,), -1, dtype=torch.int32, device="cuda")
    _abi.check(_call(Z, 100, 3, seeds))            # the first call in this context looks the array up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    reserved0 = torch.cuda.memory_reserved()
    _abi.check(_call(Z, 100, 7, seeds))
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0 and torch.cuda.memory_reserved() == reserved0
    assert np.array_equal(seeds.cpu().numpy(), api.kmeanspp(Z, 100, 7).cpu().numpy())


def test_noalloc_at_its_largest_n(cuda):
    # RAFTGP_NOALLOC_MAX_N points fill the static scratch up to its layout margin
    Z = _unit_rows(MAX_N, 32, 5, torch.float32)
    got = _noalloc(Z, 64, 11).cpu().numpy()
    ref = api.kmeanspp(Z, 64, 11).cpu().numpy()
    assert np.array_equal(got, ref) and len(set(got.tolist())) == 64
    del Z
    torch.cuda.empty_cache()


def test_noalloc_rejects_more_points_than_its_scratch_holds(cuda):
    Z = _unit_rows(64, 64, 3, torch.float32)
    seeds = torch.empty(4, dtype=torch.int32, device="cuda")
    n_too_big = MAX_N + 1      # rejected on the host before any work
    st = _abi.lib().raftgp_kmeanspp_noalloc(C.c_void_p(Z.data_ptr()), n_too_big, 64, 0, 4, 1,
                                            C.c_void_p(seeds.data_ptr()), None)
    assert st == _abi.EUNSUPPORTED
    assert b"RAFTGP_NOALLOC_MAX_N" in _abi.lib().raftgp_last_error()
