"""Streaming updates (Section III-D): after each batch of new edges the stream's graph equals
the host-built graph with those edges, its embedding equals a full FP32 embedding of the new
graph bit for bit (and the FP64 oracle's to 1e-4), only the affected rows were recomputed,
and malformed batches leave the stream unchanged."""
import numpy as np
import pytest
import torch

import oracle
from conftest import ragged_graph, rel_fro
from inputs.dcsbm import from_edges, workload
from paper_2312_01560_gb300 import api

pytestmark = pytest.mark.gpu


def _edges(g):
    rp = np.asarray(g.row_ptr, dtype=np.int64)
    src = np.repeat(np.arange(g.n), np.diff(rp))
    col = np.asarray(g.col, dtype=np.int64)
    keep = src < col
    return src[keep], col[keep]


def _new_edges(rng, g, present, m, hub=None, hub_extra=0):
    out = set()
    while len(out) < m:
        u, v = (int(x) for x in rng.integers(0, g.n, 2))
        a, b = min(u, v), max(u, v)
        if a != b and (a, b) not in present and (a, b) not in out:
            out.add((a, b))
    if hub is not None:
        for v in rng.permutation(g.n):
            if len(out) >= m + hub_extra:
                break
            a, b = min(hub, int(v)), max(hub, int(v))
            if a != b and (a, b) not in present and (a, b) not in out:
                out.add((a, b))
    e = np.array(sorted(out), dtype=np.int64)
    return e[:, 0], e[:, 1]


@pytest.mark.parametrize("case", ["ragged", "dcsbm-2k"])
def test_updates_equal_full_embedding(cuda, case):
    g = ragged_graph(4) if case == "ragged" else workload(case)
    dims = (64, 64, 32)
    st = api.Stream(api.DeviceGraph.from_host(g, cuda), dims=dims, seed=3)
    u0, v0 = _edges(g)
    present = set(zip(u0.tolist(), v0.tolist()))
    deg = np.diff(np.asarray(g.row_ptr))
    # a node just below the 256-neighbour split of the gathers, pushed above it by the updates
    hub = int(np.argmin(np.abs(deg - 250)))
    rng = np.random.default_rng(8)
    us, vs = [u0], [v0]
    for step, (m, extra) in enumerate([(1, 0), (40, 12), (300, 0)]):
        u, v = _new_edges(rng, g, present, m, hub if extra else None, extra)
        present |= set(zip(u.tolist(), v.tolist()))
        us.append(u)
        vs.append(v)
        aff = st.add_edges(torch.as_tensor(u, device=cuda), torch.as_tensor(v, device=cuda))
        ref = from_edges(g.n, np.concatenate(us), np.concatenate(vs))
        sg = st.graph()
        assert np.array_equal(sg.row_ptr.cpu().numpy(), ref.row_ptr)
        assert np.array_equal(sg.col.cpu().numpy(), ref.col)
        Z = st.embedding()
        full = api.embed(api.DeviceGraph.from_host(ref, cuda, row_ptr_bits=64), "ncut", dims, "f32", seed=3)
        torch.cuda.synchronize()
        print(f"{case} update {step}: {len(u)} edges, recomputed rows per stage {aff} of {g.n}")
        assert torch.equal(Z, full)
        assert all(a <= b for a, b in zip(aff, aff[1:])) and aff[-1] <= g.n
        assert aff[0] >= len(set(u.tolist()) | set(v.tolist()))
    _, Z_o = oracle.embed(ref, "ncut", dims, seed=3)
    assert rel_fro(Z.cpu().numpy(), Z_o) <= 1e-4


def test_one_edge_touches_a_neighbourhood(cuda):
    g = workload("dcsbm-50k")
    st = api.Stream(api.DeviceGraph.from_host(g, cuda), dims=(64, 32), seed=1)
    present = set(zip(*(x.tolist() for x in _edges(g))))
    u, v = _new_edges(np.random.default_rng(1), g, present, 1)
    aff = st.add_edges(torch.as_tensor(u, device=cuda), torch.as_tensor(v, device=cuda))
    print(f"one edge on dcsbm-50k: recomputed rows per stage {aff}")
    assert aff[0] < aff[1] < g.n


def test_malformed_batches_leave_the_stream_unchanged(cuda):
    g = workload("dcsbm-1k")
    st = api.Stream(api.DeviceGraph.from_host(g, cuda), dims=(64, 64, 32), seed=2)
    Z0 = st.embedding()
    rp0 = st.graph().row_ptr.clone()
    u0, v0 = _edges(g)
    t = lambda a: torch.as_tensor(np.asarray(a), device=cuda)
    for u, v in [([int(u0[0])], [int(v0[0])]),          # already present
                 ([1, 1], [5, 5]),                      # listed twice
                 ([7], [7]),                            # a self loop
                 ([3], [g.n])]:                         # outside [0, n)
        present = set(zip(u0.tolist(), v0.tolist()))
        if (u, v) == ([1, 1], [5, 5]) and ((1, 5) in present):
            u, v = [2, 2], [int(g.n - 1), int(g.n - 1)]
        with pytest.raises(api._abi.RaftgpError, match="EINVAL"):
            st.add_edges(t(u), t(v))
    assert torch.equal(st.embedding(), Z0)
    assert torch.equal(st.graph().row_ptr, rp0)


def test_modularity_operators_are_not_streamed(cuda):
    g = workload("dcsbm-1k")
    with pytest.raises(api._abi.RaftgpError, match="EUNSUPPORTED"):
        api.Stream(api.DeviceGraph.from_host(g, cuda), dims=(64, 32), op="mod_full")
    with pytest.raises(api._abi.RaftgpError, match="EUNSUPPORTED"):
        api.Stream(api.DeviceGraph.from_host(g, cuda), dims=(64, 32), dtype="bf16")
