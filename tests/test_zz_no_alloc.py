"""The allocation-free k-means++ entry point (raftgp_kmeanspp_noalloc) against the
workspace entry point (raftgp_kmeanspp), through the C ABI.

raftgp_kmeanspp_noalloc exists for callers that cannot allocate device memory (a plugin in
another program's CUDA context whose allocator owns the device memory, or a process that
reserves all its device memory up front); it keeps its scratch in a static device array.
Seeds are integers, so the two entry points must agree exactly; two calls in a row check
that the shared array's leftover contents from one call do not leak into the next.  This file
runs last (pytest collects it after the others) and also passes alone in a fresh process."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2312_01560_gb300 import _abi, api

pytestmark = pytest.mark.gpu


def _noalloc(Z, K, seed):
    n, d = Z.shape
    code = 1 if Z.dtype == torch.bfloat16 else 0
    seeds = torch.full((K,), -1, dtype=torch.int32, device=Z.device)
    st = _abi.lib().raftgp_kmeanspp_noalloc(C.c_void_p(Z.data_ptr()), n, d, code, K, seed,
                                            C.c_void_p(seeds.data_ptr()),
                                            C.c_void_p(torch.cuda.current_stream().cuda_stream))
    _abi.check(st)
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


def test_noalloc_rejects_more_points_than_its_scratch_holds(cuda):
    Z = _unit_rows(64, 64, 3, torch.float32)
    seeds = torch.empty(4, dtype=torch.int32, device="cuda")
    n_too_big = 4_500_001      # RAFTGP_NOALLOC_MAX_N + 1: rejected on the host before any work
    st = _abi.lib().raftgp_kmeanspp_noalloc(C.c_void_p(Z.data_ptr()), n_too_big, 64, 0, 4, 1,
                                            C.c_void_p(seeds.data_ptr()), None)
    assert st == _abi.EUNSUPPORTED
    assert b"RAFTGP_NOALLOC_MAX_N" in _abi.lib().raftgp_last_error()
