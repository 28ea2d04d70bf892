"""Failure detection without a GPU fault: a bounded device wait that runs out is reported as
RAFTGP_ETIMEOUT, and the context stays usable.  The test hook makes one block of the
persistent k-means++ kernel leave without arriving at the grid barrier, so the other
blocks' wait (2 s limit) gives up, raises the abort word and returns."""
import numpy as np
import pytest
import torch

import oracle
from inputs.dcsbm import workload
from paper_2312_01560_gb300 import api, _abi

pytestmark = pytest.mark.gpu


def test_seeding_barrier_timeout_is_reported_and_context_survives(cuda):
    g = workload("dcsbm-1k")
    _, Z = oracle.embed(g, "ncut", (64, 64, 32), seed=1)
    dg = api.DeviceGraph.from_host(g, cuda)
    Zd = torch.tensor(Z.astype(np.float32), device=cuda)
    api.debug_seed_skip_block(1)
    try:
        with pytest.raises(_abi.RaftgpError) as e:
            api.select(dg, Zd, kmin=2, kmax=12, grid=0, iters=5)
        assert e.value.status == _abi.ETIMEOUT
    finally:
        api.debug_seed_skip_block(-1)
    torch.cuda.synchronize()
    # the same call again, hook off: it completes and agrees with the oracle's seeds
    lab, rep = api.select(dg, Zd, kmin=2, kmax=12, grid=0, iters=5)
    lab = lab.cpu().numpy()
    assert 0 <= lab.min() and lab.max() < rep["k"]
    seeds = api.kmeanspp(Zd, 12, seed=2).cpu().numpy()
    assert np.array_equal(seeds, oracle.kmeanspp(Z.astype(np.float32).astype(np.float64), 12, 2,
                                                 fp32_decision=True))
