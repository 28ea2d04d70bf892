"""Streaming update of Algorithm 1 (Section III-D): after a batch of new edges only the sets of
the recursion tree that hold a changed node are partitioned again.  With the literal reading of
Eq. 7 (2e = the G-degree sum of U) the update must equal a full Algorithm 1 run on the new graph
and embedding, labels, block count and leaf ids alike, and the full run equals the FP64 oracle
(oracle/hier.py) on the new graph.  A call that flags no node keeps the previous tree whatever
embedding it is given; a call that flags every node is a full run."""
import numpy as np
import pytest
import torch

from inputs.dcsbm import Graph, dcsbm
from oracle import hier
from paper_2312_01560_gb300 import api
from paper_2312_01560_gb300.metrics import nmi

pytestmark = pytest.mark.gpu


def _graph():
    return dcsbm(1500, 6, alpha=5.0, gamma=2.5, dmin=8, dmax=60, mean_degree=24, ratio=12.0, seed=31)


def _new_edges(g, m, seed):
    rng = np.random.default_rng(seed)
    rp = np.asarray(g.row_ptr, dtype=np.int64)
    src = np.repeat(np.arange(g.n), np.diff(rp))
    present = set(zip(src.tolist(), np.asarray(g.col).tolist()))
    out = set()
    while len(out) < m:
        u, v = (int(x) for x in rng.integers(0, g.n, 2))
        a, b = min(u, v), max(u, v)
        if a != b and (a, b) not in present and (a, b) not in out:
            out.add((a, b))
    e = np.array(sorted(out), dtype=np.int64)
    return e[:, 0], e[:, 1]


def _host(dg, planted, k):
    return Graph(n=dg.n, row_ptr=dg.row_ptr.cpu().numpy().astype(np.int64), col=dg.col.cpu().numpy().astype(np.int32),
                 planted=planted, k_planted=k)


@pytest.mark.parametrize("reading", ["literal", "global"])
@pytest.mark.parametrize("m", [1, 6])
def test_streaming_update_equals_a_full_run(cuda, reading, m):
    g = _graph()
    dg = api.DeviceGraph.from_host(g, cuda)
    st = api.Stream(dg, dims=(64, 64, 32), seed=1)
    Z0 = st.embedding()
    lab0, k0, leaf0 = api.select_bisect(dg, Z0, reading=reading, return_leaf=True)
    src, dst = _new_edges(g, m, seed=m)
    st.add_edges(torch.tensor(src), torch.tensor(dst))
    g1 = st.graph()
    Z1 = st.embedding()
    changed = (Z1 != Z0).any(dim=1)
    changed[torch.tensor(src, device=cuda)] = True
    changed[torch.tensor(dst, device=cuda)] = True
    lab1, k1, leaf1 = api.select_bisect_update(g1, Z1, lab0, k0, leaf0, changed, reading=reading)
    labF, kF, leafF = api.select_bisect(g1, Z1, reading=reading, return_leaf=True)
    a = nmi(lab1.cpu().numpy(), labF.cpu().numpy())
    print(f"{reading}, {m} new edges: {int(changed.sum())} changed nodes; K old {k0} update {k1} full {kF}; "
          f"NMI(update, full) {a:.4f}")
    if reading == "literal":
        assert k1 == kF and torch.equal(lab1, labF) and torch.equal(leaf1, leafF)
        # the full run on the new graph is the oracle's
        ref, kr = hier.bisect(_host(g1, g.planted, g.k_planted), Z1.cpu().numpy(), seed=2, reading="literal")
        assert kr == kF and np.array_equal(ref, labF.cpu().numpy())
    else:
        assert a >= 0.9


def test_update_without_changed_nodes_keeps_the_tree(cuda):
    g = _graph()
    dg = api.DeviceGraph.from_host(g, cuda)
    Z = api.embed(dg, "ncut", (64, 64, 32), "f32", seed=1)
    lab0, k0, leaf0 = api.select_bisect(dg, Z, return_leaf=True)
    # an unrelated embedding: nothing is re-partitioned when no node is flagged
    Zr = torch.nn.functional.normalize(torch.randn_like(Z), dim=1)
    none = torch.zeros(g.n, dtype=torch.uint8, device=cuda)
    lab1, k1, leaf1 = api.select_bisect_update(dg, Zr, lab0, k0, leaf0, none)
    assert k1 == k0 and torch.equal(lab1, lab0) and torch.equal(leaf1, leaf0)
    # every node flagged: a full run on that embedding
    every = torch.ones(g.n, dtype=torch.uint8, device=cuda)
    lab2, k2, leaf2 = api.select_bisect_update(dg, Zr, lab0, k0, leaf0, every)
    labF, kF, leafF = api.select_bisect(dg, Zr, return_leaf=True)
    assert k2 == kF and torch.equal(lab2, labF) and torch.equal(leaf2, leafF)


def test_update_rejects_missing_previous_result(cuda):
    g = _graph()
    dg = api.DeviceGraph.from_host(g, cuda)
    Z = api.embed(dg, "ncut", (64, 64, 32), "f32", seed=1)
    lab0, k0, leaf0 = api.select_bisect(dg, Z, return_leaf=True)
    with pytest.raises(api._abi.RaftgpError):
        api.select_bisect_update(dg, Z, lab0, 0, leaf0, torch.zeros(g.n, dtype=torch.uint8, device=cuda))


def test_streaming_update_on_a_sparse_graph_reuses_the_tree(cuda):
    # one GCN layer on a sparse graph: the rows a new edge changes are a small neighbourhood,
    # so most of the tree is kept, and the result still equals a full run (literal reading)
    g = dcsbm(20000, 20, alpha=5.0, gamma=2.5, dmin=3, dmax=30, mean_degree=6, ratio=8.0, seed=7)
    dg = api.DeviceGraph.from_host(g, cuda)
    st = api.Stream(dg, dims=(64, 32), seed=1)
    Z0 = st.embedding()
    lab0, k0, leaf0 = api.select_bisect(dg, Z0, return_leaf=True)
    src, dst = _new_edges(g, 2, seed=11)
    st.add_edges(torch.tensor(src), torch.tensor(dst))
    g1 = st.graph()
    Z1 = st.embedding()
    changed = (Z1 != Z0).any(dim=1)
    changed[torch.tensor(src, device=cuda)] = True
    changed[torch.tensor(dst, device=cuda)] = True
    nch = int(changed.sum())
    lab1, k1, leaf1 = api.select_bisect_update(g1, Z1, lab0, k0, leaf0, changed)
    labF, kF, leafF = api.select_bisect(g1, Z1, return_leaf=True)
    kept = int((leaf1 == leaf0).sum())
    print(f"sparse: {nch} of {g.n} nodes changed; K old {k0} new {k1}; {kept} nodes keep their old leaf")
    assert nch < g.n // 4
    assert k1 == kF and torch.equal(lab1, labF) and torch.equal(leaf1, leafF)
