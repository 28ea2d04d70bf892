"""GPU embedding (Eq. 5 projection, Eq. 6 GCN layers) against the FP64 oracle, element by
element.  Bar: FP32 storage within 1e-4 relative Frobenius error of the oracle (expected
~1e-6: FP32 rounding plus single-precision log/sincos in the Gaussian draws); BF16 storage
is reported and held to a loose drift bound."""
import numpy as np
import pytest
import torch

import oracle
from conftest import ragged_graph, rel_fro
from inputs import small
from inputs.dcsbm import workload
from paper_2312_01560_gb300 import api

pytestmark = pytest.mark.gpu


def _np(t):
    return t.float().cpu().numpy()


@pytest.mark.parametrize("op", ["ncut", "mod_full", "mod_reduced"])
@pytest.mark.parametrize("bits", [32, 64])
def test_embed_fp32_matches_oracle(cuda, op, bits):
    g = workload("dcsbm-1k")
    dg = api.DeviceGraph.from_host(g, cuda, row_ptr_bits=bits)
    dims = (64, 64, 32)
    Z, st = api.embed(dg, op, dims, "f32", seed=1, return_stages=True)
    Y_o, Z_o = oracle.embed(g, op, dims, seed=1)
    assert rel_fro(_np(st[0]), Y_o) <= 1e-5
    Z1_o = oracle.gcn_layer(g, Y_o, oracle.gcn_weight(1, 64, 64, 1))
    assert rel_fro(_np(st[1]), Z1_o) <= 1e-5
    assert rel_fro(_np(Z), Z_o) <= 1e-4
    assert np.array_equal(_np(st[2]), _np(Z))


@pytest.mark.parametrize("op", ["ncut", "mod_full", "mod_reduced"])
def test_embed_ragged_graph(cuda, op):
    g = ragged_graph(1)
    dg = api.DeviceGraph.from_host(g, cuda)
    dims = (128, 128, 64)
    Z, st = api.embed(dg, op, dims, "f32", seed=5, return_stages=True)
    Y_o, Z_o = oracle.embed(g, op, dims, seed=5)
    assert rel_fro(_np(st[0]), Y_o) <= 1e-5
    assert rel_fro(_np(Z), Z_o) <= 1e-4
    iso = np.flatnonzero(np.diff(g.row_ptr) == 0)
    assert iso.size >= 7
    if op != "mod_full":
        assert np.abs(_np(st[0])[iso]).max() == 0.0      # isolated rows of M and Q-tilde are empty


@pytest.mark.parametrize("dims", [(32, 32), (64, 128, 32), (128, 64, 64, 32)])
def test_embed_widths_and_depths(cuda, dims):
    g = workload("dcsbm-1k", seed=2)
    dg = api.DeviceGraph.from_host(g, cuda)
    Z = api.embed(dg, "mod_full", dims, "f32", seed=3)
    _, Z_o = oracle.embed(g, "mod_full", dims, seed=3)
    assert rel_fro(_np(Z), Z_o) <= 1e-4


def test_embed_given_theta_and_weights(cuda):
    g = small.ring_of_cliques(10, 12)
    dg = api.DeviceGraph.from_host(g, cuda)
    rng = np.random.default_rng(0)
    th = rng.normal(size=(g.n, 32)) / np.sqrt(32)
    W = [rng.normal(size=(32, 64)) * 0.2, rng.normal(size=(64, 32)) * 0.2]
    Z = api.embed(dg, "ncut", (32, 64, 32), "f32", theta=torch.tensor(th), W=[torch.tensor(w) for w in W])
    _, Z_o = oracle.embed(g, "ncut", (32, 64, 32), theta_in=th, W_in=W)
    assert rel_fro(_np(Z), Z_o) <= 1e-5


def test_embed_rows_are_unit_norm_and_mod_columns_vanish(cuda):
    g = workload("dcsbm-50k")
    dg = api.DeviceGraph.from_host(g, cuda)
    Z, st = api.embed(dg, "mod_full", (128, 128, 64), "f32", seed=1, return_stages=True)
    Y = st[0].double()
    colsum = Y.sum(0).abs().max().item()
    assert colsum <= 1e-5 * Y.abs().sum(0).max().item()          # 1^T Q = 0
    norms = Z.double().norm(dim=1)
    deg = np.diff(g.row_ptr)
    ok = torch.tensor(deg > 0, device=cuda) | (norms > 0)
    assert (norms[ok] - 1).abs().max().item() < 1e-5


def test_embed_50k_matches_oracle(cuda):
    g = workload("dcsbm-50k")
    dg = api.DeviceGraph.from_host(g, cuda)
    Z = api.embed(dg, "ncut", (128, 128, 64), "f32", seed=1)
    _, Z_o = oracle.embed(g, "ncut", (128, 128, 64), seed=1)
    assert rel_fro(_np(Z), Z_o) <= 1e-4


@pytest.mark.parametrize("op", ["ncut", "mod_full"])
def test_embed_bf16_drift(cuda, op):
    g = workload("dcsbm-1k")
    dg = api.DeviceGraph.from_host(g, cuda)
    dims = (64, 64, 32)
    Z, st = api.embed(dg, op, dims, "bf16", seed=1, return_stages=True)
    Y_o, Z_o = oracle.embed(g, op, dims, seed=1)
    drift = [rel_fro(_np(st[0]), Y_o), rel_fro(_np(st[1]), oracle.gcn_layer(g, Y_o, oracle.gcn_weight(1, 64, 64, 1))),
             rel_fro(_np(Z), Z_o)]
    print(f"bf16 per-stage rel-Frobenius drift ({op}): Y {drift[0]:.2e}  Z1 {drift[1]:.2e}  Z {drift[2]:.2e}")
    assert max(drift) < 5e-2


def test_embed_is_deterministic(cuda):
    g = workload("dcsbm-1k")
    dg = api.DeviceGraph.from_host(g, cuda)
    a = api.embed(dg, "mod_full", (64, 64, 32), "f32", seed=4)
    b = api.embed(dg, "mod_full", (64, 64, 32), "f32", seed=4)
    assert torch.equal(a, b)


def test_malformed_graph_is_rejected(cuda):
    g = workload("dcsbm-1k")
    dg = api.DeviceGraph.from_host(g, cuda)
    bad = dg.col.clone()
    bad[17] = g.n                      # column index out of range
    with pytest.raises(api._abi.RaftgpError, match="EINVAL"):
        api.embed(api.DeviceGraph(g.n, dg.row_ptr, bad), "ncut", (64, 64, 32))
    bad = dg.col.clone()
    r0 = int(g.row_ptr[5])
    bad[r0] = 5                        # a self loop
    with pytest.raises(api._abi.RaftgpError, match="EINVAL"):
        api.embed(api.DeviceGraph(g.n, dg.row_ptr, bad), "ncut", (64, 64, 32))


def test_workspace_too_small(cuda):
    import ctypes as C
    g = workload("dcsbm-1k")
    dg = api.DeviceGraph.from_host(g, cuda)
    o = api.embed_opts("ncut", (64, 64, 32))
    csr = dg.csr()
    Z = torch.empty((g.n, 32), device=cuda)
    ws = torch.empty(1024, dtype=torch.uint8, device=cuda)
    st = api.lib().raftgp_embed(C.byref(csr), C.byref(o), C.c_void_p(Z.data_ptr()), C.c_void_p(ws.data_ptr()), 1024,
                                None)
    assert st == api._abi.ENOMEM


def _bf16(a):
    """Round to BF16 (nearest even) as the kernels store it."""
    return torch.as_tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


@pytest.mark.parametrize("graph", ["ragged", "dcsbm-50k"])
@pytest.mark.parametrize("op,dims", [("mod_full", (128, 128, 64)), ("ncut", (64, 64, 32))])
def test_embed_bf16_gathers_match_oracle(cuda, graph, op, dims):
    """The BF16 gathers (projection and each GCN layer) against the oracle fed the same BF16
    inputs the kernels read: Theta as stored (rounded after the NCut column scale), and for
    each GCN layer the previous stage's BF16 output through W (rounded as the dense layer
    stores it).  Bound: the projection element by element within 2^-8 relative (one BF16
    rounding of the output) plus 1e-4 of the RMS (FP32 accumulation) plus two BF16 ulps of
    the row's largest stored term (the kernel scales Theta by a single-precision reciprocal
    square root before rounding, so a stored term can sit one ulp from the one rebuilt here;
    a missing or extra neighbour is a whole term, far above this); each GCN row within
    6e-3 of the unit-norm oracle row."""
    g = ragged_graph(3) if graph == "ragged" else workload(graph)
    dg = api.DeviceGraph.from_host(g, cuda)
    L = dims[0]
    th = oracle.theta(g.n, L, 3)
    Z, st = api.embed(dg, op, dims, "bf16", seed=3, theta=torch.as_tensor(th, dtype=torch.float32),
                      return_stages=True)
    torch.cuda.synchronize()
    deg = np.diff(np.asarray(g.row_ptr, dtype=np.int64)).astype(np.float64)
    if op == "ncut":
        rs32 = np.where(deg > 0, 1.0 / np.sqrt(deg.astype(np.float32)), 0).astype(np.float32)
        stored = _bf16(th.astype(np.float32) * rs32[:, None])
        th_eff = np.where(deg[:, None] > 0, stored * np.sqrt(np.maximum(deg, 1))[:, None], 0.0)
    else:
        th_eff = _bf16(th)
    Y_ref = oracle.project(g, op, th_eff)
    Y = _np(st[0]).astype(np.float64)
    rms = np.sqrt(np.mean(Y_ref ** 2))
    tol = 2.0 ** -8 * np.abs(Y_ref) + 1e-4 * rms
    if op == "ncut":
        rp = np.asarray(g.row_ptr, dtype=np.int64)
        col = np.asarray(g.col, dtype=np.int64)
        big = np.zeros_like(Y_ref)
        nz = np.flatnonzero(deg > 0)
        big[nz] = np.maximum.reduceat(np.abs(stored)[col], rp[:-1][nz], axis=0)
        tol += 2 * 2.0 ** -8 * (rs32[:, None] * big)
    bad = np.abs(Y - Y_ref) > tol
    print(f"{graph} {op} projection: max |error| / bound {np.max(np.abs(Y - Y_ref) / tol):.3f}")
    assert not bad.any(), (int(bad.sum()), np.argwhere(bad)[:5])
    rsh = 1.0 / np.sqrt(deg + 1.0)
    for k in range(1, len(dims)):
        W = oracle.gcn_weight(k, dims[k - 1], dims[k], 3)
        prev = _np(st[k - 1]).astype(np.float64)
        P = _bf16(rsh[:, None] * (prev @ W))        # what the gather reads: rsh_j (Z W)_j
        ref = oracle.gcn_layer(g, P / rsh[:, None], np.eye(dims[k]))
        got = _np(st[k]).astype(np.float64)
        row_err = np.linalg.norm(got - ref, axis=1)
        print(f"{graph} {op} layer {k}: max row error {row_err.max():.2e}, mean {row_err.mean():.2e}")
        assert row_err.max() <= 6e-3, (k, int(np.argmax(row_err)), row_err.max())


@pytest.mark.parametrize("dtype,tol", [("f32", 1e-5), ("bf16", 6e-3)])
@pytest.mark.parametrize("op", ["ncut", "mod_full", "mod_reduced"])
def test_embed_without_gcn_layers_matches_oracle(cuda, op, dtype, tol):
    # the "w/o Emb" ablation: no GCN layer, Z = rownorm(Y) on both sides
    g = workload("dcsbm-1k")
    dg = api.DeviceGraph.from_host(g, cuda)
    Z = api.embed(dg, op, (64,), dtype, seed=3)
    _, Z_o = oracle.embed(g, op, (64,), seed=3)
    assert rel_fro(_np(Z), Z_o) <= tol
    lab, rep = api.select(dg, Z, kmin=2, kmax=20)
    lab = lab.cpu().numpy()
    _, _, mod, _ = oracle.score(g, lab, int(lab.max()) + 1)
    assert [c[1] for c in rep["cands"] if c[0] == rep["k"]][0] == mod
