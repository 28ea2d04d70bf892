"""Degenerate inputs end to end against the FP64 oracle.

- A graph without edges: every embedding row is zero (the projection has no neighbours, the
  rank-one term of the full modularity operator is dropped with 2e = 0, tanh(0) = 0 and a zero
  row stays zero), so k-means++ takes its all-duplicates rule and every label is a tie.
- A star: every leaf's row is the same bit pattern on both sides (the same operations on the
  same inputs), so the seeding meets duplicate points and the assignment meets exact ties.
- A single node, and a K range beyond N (clamped to N: the last candidate puts every node in
  a block of its own).

Identical rows give identical scores in any precision, so for the first two graphs the
labels, K* and every candidate's modularity must equal the oracle's exactly, in the FP32 form
and in the BF16 form with either tensor-core engine."""
import numpy as np
import pytest

import oracle
from inputs import small
from paper_2312_01560_gb300 import api
from paper_2312_01560_gb300.metrics import nmi

pytestmark = pytest.mark.gpu

FORMS = [("f32", "ffma"), ("bf16", "tc8"), ("bf16", "tc")]
DIMS = (64, 64, 32)


def _graph(name):
    return small.edgeless(300) if name == "edgeless" else small.star(199)


@pytest.mark.parametrize("dtype,assign", FORMS)
@pytest.mark.parametrize("op", ["ncut", "mod_full"])
@pytest.mark.parametrize("name", ["edgeless", "star"])
def test_degenerate_graph_partition_equals_oracle(cuda, name, op, dtype, assign):
    g = _graph(name)
    dg = api.DeviceGraph.from_host(g, cuda)
    labels, rep = api.partition(dg, op=op, dims=DIMS, dtype=dtype, assign=assign, kmin=2, kmax=12, grid=0, iters=50)
    ref = oracle.partition(g, op, DIMS, kmin=2, kmax=12, grid=0, T=50)
    lab = labels.cpu().numpy()
    assert rep["k"] == ref["k"]
    assert np.array_equal(lab, ref["labels"])
    gpu_mod = sorted((int(c[0]), float(c[1])) for c in rep["cands"])
    ref_mod = sorted((int(c[0]), float(c[1])) for c in ref["cands"])
    assert gpu_mod == ref_mod
    if name == "edgeless":
        assert rep["k"] == 2 and not lab.any()            # every candidate scores 0: the smallest K wins
    else:
        assert rep["k"] == 2 and lab[0] != lab[1] and np.all(lab[1:] == lab[1])   # the hub alone


@pytest.mark.parametrize("dtype,assign", FORMS)
def test_single_node(cuda, dtype, assign):
    g = small.edgeless(1)
    dg = api.DeviceGraph.from_host(g, cuda)
    labels, rep = api.partition(dg, op="ncut", dims=DIMS, dtype=dtype, assign=assign, kmin=1, kmax=1, grid=0, iters=50)
    assert rep["k"] == 1
    assert labels.cpu().tolist() == [0]


@pytest.mark.parametrize("dtype,assign", FORMS)
def test_k_range_beyond_n_is_clamped(cuda, dtype, assign):
    g = small.ring_of_cliques(5, 6)                       # 30 nodes
    dg = api.DeviceGraph.from_host(g, cuda)
    labels, rep = api.partition(dg, op="ncut", dims=DIMS, dtype=dtype, assign=assign, kmin=2, kmax=40, grid=0,
                                iters=50)
    ref = oracle.partition(g, "ncut", DIMS, kmin=2, kmax=40, grid=0, T=50)
    ks = sorted(int(c[0]) for c in rep["cands"])
    assert ks == list(range(2, 31)) == sorted(int(c[0]) for c in ref["cands"])
    assert rep["k"] == ref["k"] == 5
    assert nmi(labels.cpu().numpy(), ref["labels"]) == pytest.approx(1.0, abs=1e-12)
    assert nmi(labels.cpu().numpy(), g.planted) == pytest.approx(1.0, abs=1e-12)
