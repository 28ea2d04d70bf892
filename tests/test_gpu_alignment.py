"""Workspaces at any address, and the 16-byte rule of the differentiation calls.

Every *_workspace_size() includes 256 bytes of slack and the library rounds the caller's
workspace pointer up to a 256-byte boundary inside it, so a workspace handed over 8 bytes past
a boundary must give the same results, bit for bit, as an aligned one (the TMA, cp.async and
16-byte accesses into workspace pieces stay aligned).  The layer arrays of the
differentiation calls are read and written in 16-byte pieces: a misaligned one is rejected
with RAFTGP_EINVAL before any launch, and so is a misaligned loss gradient dZ."""
import numpy as np
import pytest
import torch

from inputs.dcsbm import workload
from paper_2312_01560_gb300 import api

pytestmark = pytest.mark.gpu


def _shift_workspaces(monkeypatch, off):
    keep = []

    def ws(nbytes, device):
        t = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        keep.append(t)
        return t[off:off + nbytes]

    monkeypatch.setattr(api, "_workspace", ws)


@pytest.mark.parametrize("dtype,assign", [("bf16", "tc8"), ("bf16", "tc"), ("f32", "ffma")])
def test_partition_with_a_shifted_workspace(cuda, monkeypatch, dtype, assign):
    g = workload("dcsbm-2k")
    dg = api.DeviceGraph.from_host(g, cuda)
    kw = dict(op="mod_full", dims=(128, 128, 64), dtype=dtype, assign=assign, kmin=2, kmax=40, grid=5)
    lab0, rep0 = api.partition(dg, **kw)
    _shift_workspaces(monkeypatch, 8)
    lab1, rep1 = api.partition(dg, **kw)
    assert torch.equal(lab0, lab1)
    assert rep0["k"] == rep1["k"]
    assert [tuple(c) for c in rep0["cands"]] == [tuple(c) for c in rep1["cands"]]


def test_diff_calls_with_a_shifted_workspace(cuda, monkeypatch):
    g = workload("dcsbm-2k")
    dg = api.DeviceGraph.from_host(g, cuda)
    rng = np.random.default_rng(3)
    H = torch.tensor(rng.normal(size=(g.n, 128)), dtype=torch.float32, device=cuda)
    W = torch.tensor(rng.normal(size=(128, 64)) * 0.1, dtype=torch.float32, device=cuda)
    dHo = torch.tensor(rng.normal(size=(g.n, 64)), dtype=torch.float32, device=cuda)
    Z = torch.nn.functional.normalize(torch.tensor(rng.normal(size=(g.n, 64)), dtype=torch.float32, device=cuda))
    mu = Z[:20].contiguous()

    def run():
        out = api.gcn_layer_forward(dg, H, W)
        dH, dW = api.gcn_layer_backward(dg, H, W, dHo)
        loss, dZ = api.softmod_loss(dg, Z, mu, 0.1)
        return out, dH, dW, loss, dZ

    a = run()
    _shift_workspaces(monkeypatch, 8)
    b = run()
    assert a[3] == b[3]
    for x, y in zip(a[:3] + a[4:], b[:3] + b[4:]):
        assert torch.equal(x, y)


def test_misaligned_layer_arrays_are_rejected(cuda):
    g = workload("dcsbm-1k")
    dg = api.DeviceGraph.from_host(g, cuda)
    W = torch.zeros((64, 64), device=cuda)
    big = torch.zeros(g.n * 64 + 1, device=cuda)
    H_odd = big[1:].view(g.n, 64)                     # contiguous, 4 bytes past a 16-byte boundary
    assert H_odd.is_contiguous() and H_odd.data_ptr() % 16 == 4
    with pytest.raises(api._abi.RaftgpError, match="16-byte"):
        api.gcn_layer_forward(dg, H_odd, W)
    plan = api.DiffPlan(dg, 64, 4)
    with pytest.raises(api._abi.RaftgpError, match="16-byte"):
        plan.layer_backward(torch.zeros((g.n, 64), device=cuda), W, H_odd)
    # the loss gradient is written in 16-byte pieces too: an odd dZ is refused before any launch
    import ctypes as C
    Z = torch.nn.functional.normalize(torch.ones((g.n, 64), device=cuda))
    mu = Z[:4].contiguous()
    loss = torch.empty((), dtype=torch.float64, device=cuda)
    st = api.lib().raftgp_diff_plan_softmod_loss(plan._h, C.c_void_p(Z.data_ptr()), 64, C.c_void_p(mu.data_ptr()), 4,
                                                 0.1, C.c_void_p(loss.data_ptr()), C.c_void_p(H_odd.data_ptr()), None)
    assert st == api._abi.EINVAL and "dZ" in api.lib().raftgp_last_error().decode()
