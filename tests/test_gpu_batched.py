"""Many graphs at once: a batch of uneven graphs partitioned by one captured plan gives every
graph exactly the result of partitioning it alone (NCut operator, FP32 engine, same seeds and
grid), and agrees with the FP64 oracle's partition; replays are deterministic; malformed
batches are rejected before any work."""
import math

import numpy as np
import pytest
import torch

import oracle
from inputs.dcsbm import batch_workload, dcsbm
from paper_2312_01560_gb300 import api
from paper_2312_01560_gb300.metrics import nmi

pytestmark = pytest.mark.gpu

DIMS = (64, 64, 32)


def _kmax(n, factor=2.0):
    return min(int(math.ceil(factor * n ** 0.35)), 128, n)


@pytest.fixture(scope="module")
def batch():
    return batch_workload(n_graphs=12, seed=17, n_lo=1000, n_hi=6000)


def test_batched_equals_single_graph_partitions(cuda, batch):
    dg, off = api.concat_graphs(batch, cuda)
    plan = api.BatchPlan(dg, off, dims=DIMS, dtype="f32", kmin=2, grid=10, iters=50, seed=2)
    labels, ks = plan.run()
    torch.cuda.synchronize()
    labels, ks = labels.cpu().numpy(), ks.cpu().numpy()
    ck, cmod, cncut, cpass = plan.candidates()
    for gi, g in enumerate(batch):
        one = api.DeviceGraph.from_host(g, cuda)
        lab1, rep1 = api.partition(one, op="ncut", dims=DIMS, dtype="f32", kmin=2, kmax=_kmax(g.n), grid=10,
                                   iters=50, assign="ffma", select_seed=2)
        assert ks[gi] == rep1["k"], gi
        assert np.array_equal(labels[off[gi]:off[gi + 1]], lab1.cpu().numpy()), gi
        mine = sorted((int(k), m, c, int(p)) for k, m, c, p in zip(ck[gi], cmod[gi], cncut[gi], cpass[gi]) if k > 0)
        theirs = sorted((int(c[0]), c[1], c[2], int(c[3])) for c in rep1["cands"])
        assert mine == theirs, gi
    plan.close()


def test_batched_agrees_with_oracle(cuda):
    # strongly planted graphs of uneven size, where the FP64 oracle's partition is a stable
    # target (on weakly planted graphs FP32 and FP64 Lloyd runs settle in different optima; the
    # batched result there equals the single-graph FP32 result, checked above)
    sub = [dcsbm(n, k, alpha=5.0, gamma=2.5, dmin=8, dmax=60, mean_degree=24, ratio=12.0, seed=30 + i)
           for i, (n, k) in enumerate([(1500, 6), (3000, 9), (2200, 7)])]
    dg, off = api.concat_graphs(sub, cuda)
    plan = api.BatchPlan(dg, off, dims=DIMS, dtype="f32", kmin=2, grid=10, iters=50, seed=2)
    labels, ks = plan.run()
    torch.cuda.synchronize()
    labels, ks = labels.cpu().numpy(), ks.cpu().numpy()
    for gi, g in enumerate(sub):
        ref = oracle.partition(g, "ncut", DIMS, kmin=2, kmax=_kmax(g.n), grid=10)
        lab = labels[off[gi]:off[gi + 1]]
        a = nmi(lab, ref["labels"])
        print(f"graph {gi} (N={g.n}): K* {ks[gi]} (oracle {ref['k']}), NMI vs oracle {a:.4f}, "
              f"vs planted {nmi(lab, g.planted):.4f}")
        assert ks[gi] == ref["k"]
        assert a >= 0.99
    plan.close()


def test_replay_is_deterministic_and_tuned(cuda, batch):
    dg, off = api.concat_graphs(batch[:6], cuda)
    plan = api.BatchPlan(dg, off, dims=DIMS, dtype="f32", kmin=2, grid=10, iters=50, seed=2)
    a = [t.clone() for t in plan.run()]
    b = [t.clone() for t in plan.run()]
    torch.cuda.synchronize()
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    t = plan.tuning()
    assert t["threads"] in (128, 256, 512) and t["points_per_thread"] in (0, 1, 2)
    assert len(t["ms"]) == 7 and all(m > 0 for m in t["ms"])
    print(f"batch tuning: {t}")
    plan.close()


def test_bf16_batch_runs(cuda, batch):
    dg, off = api.concat_graphs(batch[:4], cuda)
    plan = api.BatchPlan(dg, off, dims=DIMS, dtype="bf16", kmin=2, grid=10, iters=50, seed=2)
    labels, ks = plan.run()
    torch.cuda.synchronize()
    ks = ks.cpu().numpy()
    for gi, g in enumerate(batch[:4]):
        assert 2 <= ks[gi] <= _kmax(g.n)
        lab = labels[off[gi]:off[gi + 1]].cpu().numpy()
        assert lab.min() >= 0 and lab.max() < ks[gi]
    plan.close()


def test_cross_graph_edge_is_rejected(cuda, batch):
    dg, off = api.concat_graphs(batch[:2], cuda)
    col = dg.col.clone()
    col[0] = int(off[1])           # a column of graph 0's first row pointing into graph 1
    bad = api.DeviceGraph(dg.n, dg.row_ptr, col)
    with pytest.raises(api._abi.RaftgpError, match="malformed"):
        api.BatchPlan(bad, off, dims=DIMS, dtype="f32")


def test_bad_offsets_are_rejected(cuda, batch):
    dg, off = api.concat_graphs(batch[:2], cuda)
    with pytest.raises(api._abi.RaftgpError):
        api.BatchPlan(dg, off[:-1], dims=DIMS, dtype="f32")


def test_every_lloyd_variant_gives_the_same_result(cuda, batch):
    # the autotuner's seven Lloyd kernels (six scalar shapes, the register-tiled kernel) differ
    # only in speed: labels, K* and every candidate's score agree bit for bit
    dg, off = api.concat_graphs(batch[:5], cuda)
    ref = None
    for v in range(1, 8):
        plan = api.BatchPlan(dg, off, dims=DIMS, dtype="f32", kmin=2, grid=10, iters=50, seed=2, lloyd_variant=v)
        labels, ks = plan.run()
        torch.cuda.synchronize()
        ck, cm, cn, cp = plan.candidates()
        used = ck > 0                                 # unused slots (k = 0) hold no result
        got = (labels.cpu().numpy(), ks.cpu().numpy(), ck, cm[used], cn[used], cp[used])
        t = plan.tuning()
        assert (t["threads"], t["points_per_thread"]) == (([128, 256, 512][(v - 1) // 2], 1 + (v - 1) % 2) if v < 7
                                                          else (256, 0))
        plan.close()
        if ref is None:
            ref = got
        else:
            for a, b in zip(ref, got):
                assert np.array_equal(a, b), v


def test_bf16_batch_equals_single_graph_selection_on_its_embedding(cuda, batch):
    # BF16 storage: every graph's model selection on the plan's own BF16 embedding equals a
    # single-graph selection (FP32 engine) on the same rows, and each chosen partition that
    # converged assigns every point to its nearest centroid (FP32 band); drift against the
    # FP32 batch is stated
    sub = batch[:6]
    dg, off = api.concat_graphs(sub, cuda)
    plan = api.BatchPlan(dg, off, dims=DIMS, dtype="bf16", kmin=2, grid=10, iters=50, seed=2)
    labels, ks = plan.run()
    torch.cuda.synchronize()
    Z = plan.embedding()
    labels, ks = labels.cpu().numpy(), ks.cpu().numpy()
    ck, cmod, cncut, cpass = plan.candidates()
    plan32 = api.BatchPlan(dg, off, dims=DIMS, dtype="f32", kmin=2, grid=10, iters=50, seed=2)
    l32, k32 = plan32.run()
    torch.cuda.synchronize()
    l32, k32 = l32.cpu().numpy(), k32.cpu().numpy()
    for gi, g in enumerate(sub):
        one = api.DeviceGraph.from_host(g, cuda)
        Zg = Z[off[gi]:off[gi + 1]].contiguous()
        lab1, rep1 = api.select(one, Zg, kmin=2, kmax=_kmax(g.n), grid=10, iters=50, assign="ffma", seed=2)
        lab = labels[off[gi]:off[gi + 1]]
        assert ks[gi] == rep1["k"] and np.array_equal(lab, lab1.cpu().numpy()), gi
        slot = [j for j in range(20) if ck[gi, j] == ks[gi]][0]
        if cpass[gi, slot] < 50:                     # converged: centroids are the label means
            z = Zg.float().cpu().numpy().astype(np.float64)
            K = int(ks[gi])
            mu = np.stack([z[lab == c].mean(0) if (lab == c).any() else np.full(z.shape[1], np.inf)
                           for c in range(K)])
            d2 = ((z[:, None, :] - mu[None]) ** 2).sum(-1)
            own = d2[np.arange(len(lab)), lab]
            assert (own <= d2.min(1) + 1e-5).all(), gi
        print(f"graph {gi} (N={g.n}): K* bf16 {ks[gi]} fp32 {k32[gi]}, NMI(bf16, fp32) "
              f"{nmi(lab, l32[off[gi]:off[gi + 1]]):.4f}, NMI vs planted bf16 {nmi(lab, g.planted):.4f} "
              f"fp32 {nmi(l32[off[gi]:off[gi + 1]], g.planted):.4f}")
    plan.close()
    plan32.close()


@pytest.mark.parametrize("dims", [DIMS, (64, 64, 64)])
@pytest.mark.parametrize("engine", ["tc8", "tc"])
def test_tensor_core_batch_matches_single_graph_tensor_core_selection(cuda, batch, engine, dims):
    # tensor-core Lloyd in the batched plan: every graph's candidates, K* and labels equal a
    # single-graph selection with the same engine on the plan's own BF16 embedding (whose final
    # labels are the FP32-nearest centroids of the last Lloyd pass, tested with the single-graph
    # engine); drift against the FP32-engine batch is stated
    sub = batch[:6]
    dg, off = api.concat_graphs(sub, cuda)
    plan = api.BatchPlan(dg, off, dims=dims, dtype="bf16", kmin=2, grid=10, iters=50, seed=2, assign=engine)
    labels, ks = plan.run()
    plan.check()
    Z = plan.embedding()
    labels, ks = labels.cpu().numpy(), ks.cpu().numpy()
    ck, cmod, cncut, cpass = plan.candidates()
    t = plan.tuning()
    assert t["points_per_thread"] == -1
    plan32 = api.BatchPlan(dg, off, dims=dims, dtype="bf16", kmin=2, grid=10, iters=50, seed=2)
    l32, k32 = plan32.run()
    plan32.check()
    l32, k32 = l32.cpu().numpy(), k32.cpu().numpy()
    for gi, g in enumerate(sub):
        one = api.DeviceGraph.from_host(g, cuda)
        Zg = Z[off[gi]:off[gi + 1]].contiguous()
        lab1, rep1 = api.select(one, Zg, kmin=2, kmax=_kmax(g.n), grid=10, iters=50, assign=engine, seed=2)
        lab = labels[off[gi]:off[gi + 1]]
        mine = sorted((int(k), m, int(p)) for k, m, p in zip(ck[gi], cmod[gi], cpass[gi]) if k > 0)
        theirs = sorted((int(c[0]), c[1], int(c[3])) for c in rep1["cands"])
        same = sum(a == b for a, b in zip(mine, theirs))
        print(f"graph {gi} (N={g.n}) {engine}: K* batch {ks[gi]} single {rep1['k']}; candidates equal {same}/"
              f"{len(theirs)}; NMI(batch, single) {nmi(lab, lab1.cpu().numpy()):.4f}; NMI vs FP32-engine batch "
              f"{nmi(lab, l32[off[gi]:off[gi + 1]]):.4f}")
        assert ks[gi] == rep1["k"] and np.array_equal(lab, lab1.cpu().numpy()), gi
        assert mine == theirs, gi
    plan.close()
    plan32.close()


def test_tensor_core_batch_needs_bf16(cuda, batch):
    dg, off = api.concat_graphs(batch[:2], cuda)
    with pytest.raises(api._abi.RaftgpError, match="BF16"):
        api.BatchPlan(dg, off, dims=DIMS, dtype="f32", assign="tc8")


def test_every_embedding_gather_shape_gives_the_same_embedding(cuda, batch):
    # the autotuner's four flat-stream gather shapes (entries per batch, staging depth) change
    # only speed: the batch's BF16 embedding is the same bits for each, and equals every
    # graph's single-graph BF16 embedding
    dg, off = api.concat_graphs(batch[:4], cuda)
    dims = (128, 128, 64)
    ref = None
    for v in range(1, 5):
        plan = api.BatchPlan(dg, off, dims=dims, dtype="bf16", kmin=2, grid=10, iters=3, seed=2, embed_variant=v)
        plan.run()
        plan.check()
        Z = plan.embedding()
        assert plan.tuning()["embed_gather_variant"] == v - 1
        plan.close()
        if ref is None:
            ref = Z
        else:
            assert torch.equal(Z.view(torch.int16), ref.view(torch.int16)), v
    for gi, g in enumerate(batch[:4]):
        one = api.DeviceGraph.from_host(g, cuda)
        Zg = api.embed(one, "ncut", dims, "bf16", seed=1)
        assert torch.equal(Zg.view(torch.int16), ref[off[gi]:off[gi + 1]].view(torch.int16)), gi
    plan = api.BatchPlan(dg, off, dims=dims, dtype="bf16", kmin=2, grid=10, iters=3, seed=2)
    t = plan.tuning()
    print(f"embedding gather tuning: {t['embed_gather_variant']} {t['embed_gather_ms']}")
    assert 0 <= t["embed_gather_variant"] <= 3 and all(m > 0 for m in t["embed_gather_ms"])
    plan.close()


def test_mod_full_batch_embedding_matches_the_oracle(cuda, batch):
    # the full modularity operator in the batched form: each graph's rank-one term from its own
    # degrees and Theta rows; the batch's BF16 embedding of each graph is within BF16 storage
    # error of the FP64 oracle's embedding of that graph alone, and close to the single-graph
    # BF16 embedding (the rank-one sums run in another order)
    from conftest import rel_fro
    sub = batch[:4]
    dg, off = api.concat_graphs(sub, cuda)
    dims = (64, 64, 32)
    plan = api.BatchPlan(dg, off, dims=dims, dtype="bf16", op="mod_full", kmin=2, grid=10, iters=50, seed=2,
                         assign="tc8")
    labels, ks = plan.run()
    plan.check()
    Z = plan.embedding().float().cpu().numpy()
    labels, ks = labels.cpu().numpy(), ks.cpu().numpy()
    for gi, g in enumerate(sub):
        _, Zo = oracle.embed(g, "mod_full", dims, seed=1)
        Zg = Z[off[gi]:off[gi + 1]]
        one = api.DeviceGraph.from_host(g, cuda)
        Z1 = api.embed(one, "mod_full", dims, "bf16", seed=1).float().cpu().numpy()
        e_or, e_one = rel_fro(Zg, Zo), rel_fro(Zg, Z1)
        lab = labels[off[gi]:off[gi + 1]]
        print(f"graph {gi} (N={g.n}): rel. error vs oracle {e_or:.2e}, vs single-graph BF16 {e_one:.2e}; "
              f"K* {ks[gi]}, NMI vs planted {nmi(lab, g.planted):.4f}")
        assert e_or <= 6e-3 and e_one <= 2e-3
        assert 2 <= ks[gi] <= _kmax(g.n) and lab.min() >= 0 and lab.max() < ks[gi]
    plan.close()


def test_mod_full_batch_needs_bf16(cuda, batch):
    dg, off = api.concat_graphs(batch[:2], cuda)
    with pytest.raises(api._abi.RaftgpError, match="BF16"):
        api.BatchPlan(dg, off, dims=DIMS, dtype="f32", op="mod_full")
