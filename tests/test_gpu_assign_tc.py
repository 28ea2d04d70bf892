"""Tensor-core (tcgen05, BF16) k-means assignment against the FP32 engine and the FP64
oracle.  The final assignment of a Lloyd run re-checks every near tie in FP32, so every
reported label must be the FP64-nearest centroid up to FP32 rounding; the Lloyd trajectory
may differ from the FP32 engine only through near ties of the BF16 product."""
import numpy as np
import pytest
import torch

import oracle
from inputs.dcsbm import workload
from paper_2312_01560_gb300 import api
from paper_2312_01560_gb300.metrics import nmi

pytestmark = pytest.mark.gpu


def _unit_rows(rng, n, d):
    z = rng.normal(size=(n, d))
    return z / np.linalg.norm(z, axis=1, keepdims=True)


def _nearest_ok(Z, labels, mu, tol=2e-5):
    Z = Z.astype(np.float64)
    mu = mu.astype(np.float64)
    zz = (Z * Z).sum(1)[:, None]
    d2 = zz - 2 * Z @ mu.T + (mu * mu).sum(1)[None, :]
    chosen = d2[np.arange(Z.shape[0]), labels]
    bad = chosen > d2.min(axis=1) + tol
    return int(bad.sum())


@pytest.mark.parametrize("engine", ["tc", "tc8"])
@pytest.mark.parametrize("d", [32, 64, 128])
@pytest.mark.parametrize("K", [7, 300, 1000])
def test_final_labels_are_exact_nearest(cuda, d, K, engine):
    rng = np.random.default_rng(d + K)
    n = 5003                                     # not a multiple of the 128-point tile
    Z = torch.tensor(_unit_rows(rng, n, d), dtype=torch.bfloat16, device=cuda)
    Zh = Z.float().cpu().numpy()
    mu0 = torch.tensor(Zh[rng.choice(n, K, replace=False)], device=cuda)
    lab, mu, passes = api.lloyd(Z, mu0, iters=8, assign=engine)
    assert _nearest_ok(Zh, lab.cpu().numpy(), mu.cpu().numpy()) == 0


@pytest.mark.parametrize("engine,min_agree", [("tc", 0.99), ("tc8", 0.97)])
@pytest.mark.parametrize("d", [32, 64])
def test_tc_lloyd_agrees_with_fp32_engine(cuda, d, engine, min_agree):
    g = workload("dcsbm-1k")
    _, Zo = oracle.embed(g, "ncut", (64, 64, d), seed=1)
    Z = torch.tensor(Zo, dtype=torch.bfloat16, device=cuda)
    Zh = Z.float().cpu().numpy()
    seeds = oracle.kmeanspp(Zh.astype(np.float64), 20, 3, fp32_decision=True)
    mu0 = torch.tensor(Zh[seeds], device=cuda)
    l_tc, mu_tc, p_tc = api.lloyd(Z, mu0, iters=50, assign=engine)
    l_ff, mu_ff, p_ff = api.lloyd(Z, mu0, iters=50, assign="ffma")
    lo, _, po = oracle.lloyd(Zh.astype(np.float64), Zh[seeds].astype(np.float64), 50)
    a = (l_tc.cpu().numpy() == lo).mean()
    b = (l_ff.cpu().numpy() == lo).mean()
    print(f"d={d}: label agreement with the FP64 oracle: {engine} {a:.4f} ffma {b:.4f}; "
          f"passes {engine} {p_tc} ffma {p_ff} oracle {po}")
    assert a >= min_agree
    assert _nearest_ok(Zh, l_tc.cpu().numpy(), mu_tc.cpu().numpy()) == 0


def test_tc_select_matches_ffma_select(cuda):
    g = workload("dcsbm-1k")
    _, Zo = oracle.embed(g, "mod_full", (64, 64, 64), seed=1)
    Z = torch.tensor(Zo, dtype=torch.bfloat16, device=cuda)
    dg = api.DeviceGraph.from_host(g, cuda)
    l1, r1 = api.select(dg, Z, kmin=2, kmax=40, assign="tc")
    l2, r2 = api.select(dg, Z, kmin=2, kmax=40, assign="ffma")
    same = sum(a[1] == b[1] for a, b in zip(r1["cands"], r2["cands"]))
    print(f"tc vs ffma: {same}/{len(r1['cands'])} candidates with identical modularity; K* {r1['k']} vs {r2['k']}")
    assert same >= 0.8 * len(r1["cands"])
    assert nmi(l1.cpu().numpy(), l2.cpu().numpy()) >= 0.98
    lab = l1.cpu().numpy()
    _, _, mod, _ = oracle.score(g, lab, int(lab.max()) + 1)
    assert [c[1] for c in r1["cands"] if c[0] == r1["k"]][0] == mod


@pytest.mark.parametrize("engine", ["tc", "tc8"])
def test_tc_partition_vs_oracle(cuda, engine):
    g = workload("dcsbm-1k")
    dg = api.DeviceGraph.from_host(g, cuda)
    lab, rep = api.partition(dg, op="ncut", dims=(64, 64, 32), dtype="bf16", kmin=2, kmax=40, assign=engine)
    ref = oracle.partition(g, "ncut", (64, 64, 32), kmin=2, kmax=40)
    a = nmi(lab.cpu().numpy(), ref["labels"])
    print(f"bf16+{engine} partition: K* {rep['k']} (oracle {ref['k']}), NMI vs oracle {a:.4f}, "
          f"vs planted {nmi(lab.cpu().numpy(), g.planted):.4f} (oracle {nmi(ref['labels'], g.planted):.4f})")
    assert a >= 0.9


@pytest.mark.parametrize("engine", ["tc", "tc8"])
def test_tc_is_deterministic(cuda, engine):
    g = workload("dcsbm-1k", seed=3)
    dg = api.DeviceGraph.from_host(g, cuda)
    a = api.partition(dg, dtype="bf16", assign=engine, kmin=2, kmax=40)
    b = api.partition(dg, dtype="bf16", assign=engine, kmin=2, kmax=40)
    assert a[1] == b[1] and torch.equal(a[0], b[0])


def test_tc_rejects_fp32_embeddings(cuda):
    Z = torch.zeros((100, 64), device=cuda)
    Z[:, 0] = 1
    with pytest.raises(api._abi.RaftgpError, match="BF16"):
        api.lloyd(Z, Z[:3].clone(), assign="tc")
