"""The differentiation form against the FP64 oracle (oracle/diff.py, pinned by central finite
differences): layer forward and backward, the relaxed modularity and its gradient, the whole
chain's weight gradients through torch.autograd, Adam, centroids, the exported weights; the
tuning loop lowers the loss and is deterministic.  Bars: FP32 forward within 1e-5 relative
Frobenius, gradients within 1e-4."""
import numpy as np
import pytest
import torch

import oracle
from conftest import ragged_graph, rel_fro
from inputs.dcsbm import workload
from oracle import diff as odiff
from paper_2312_01560_gb300 import api, diff

pytestmark = pytest.mark.gpu


def _np(t):
    return t.detach().double().cpu().numpy()


def _graphs():
    return [("ragged", ragged_graph()), ("dcsbm-2k", workload("dcsbm-2k"))]


@pytest.mark.parametrize("name,g", _graphs())
@pytest.mark.parametrize("lin,lout", [(64, 32), (128, 128), (32, 64)])
def test_layer_forward_and_backward_match_oracle(cuda, name, g, lin, lout):
    rng = np.random.default_rng(lin + lout)
    dg = api.DeviceGraph.from_host(g, cuda)
    H = torch.tensor(rng.normal(size=(g.n, lin)), dtype=torch.float32, device=cuda)
    W = torch.tensor(rng.normal(size=(lin, lout)) * np.sqrt(2 / (lin + lout)), dtype=torch.float32, device=cuda)
    dHo = torch.tensor(rng.normal(size=(g.n, lout)), dtype=torch.float32, device=cuda)
    Ah = odiff.a_hat(g)
    Hn, Wn = _np(H), _np(W)
    Ho, T, r = odiff.layer_forward(Ah, Hn, Wn)
    out = api.gcn_layer_forward(dg, H, W)
    assert rel_fro(_np(out), Ho) <= 1e-5
    dH, dW = api.gcn_layer_backward(dg, H, W, dHo)
    dH_o, dW_o = odiff.layer_backward(Ah, Hn, Wn, T, r, Ho, _np(dHo))
    assert rel_fro(_np(dW), dW_o) <= 1e-4
    assert rel_fro(_np(dH), dH_o) <= 1e-4


@pytest.mark.parametrize("K,d,tau", [(11, 32, 0.1), (80, 64, 0.1), (128, 128, 0.5), (3, 64, 2.0)])
def test_softmod_loss_and_gradient_match_oracle(cuda, K, d, tau):
    g = workload("dcsbm-2k")
    rng = np.random.default_rng(K)
    Z = rng.normal(size=(g.n, d))
    Z /= np.linalg.norm(Z, axis=1, keepdims=True)
    mu = Z[rng.choice(g.n, K, replace=False)] + 0.05 * rng.normal(size=(K, d))
    dg = api.DeviceGraph.from_host(g, cuda)
    Zt = torch.tensor(Z, dtype=torch.float32, device=cuda)
    mut = torch.tensor(mu, dtype=torch.float32, device=cuda)
    loss, dZ = api.softmod_loss(dg, Zt, mut, tau)
    lo, dZo = odiff.softmod_grad(g, _np(Zt), _np(mut), tau)
    assert abs(loss - lo) <= 1e-5 * max(abs(lo), 1e-3)
    assert rel_fro(_np(dZ), dZo) <= 1e-4


def test_chain_gradient_matches_oracle(cuda):
    g = workload("dcsbm-2k")
    dg = api.DeviceGraph.from_host(g, cuda)
    dims = (64, 64, 32)
    _, st = api.embed(dg, op="ncut", dims=dims, dtype="f32", seed=1, return_stages=True)
    Y = st[0]
    Ws = [api.gcn_weights(k, dims[k - 1], dims[k], 1, cuda) for k in range(1, len(dims))]
    lab, rep = api.partition(dg, op="ncut", dims=dims, dtype="f32", kmin=2, kmax=16)
    Z = diff.chain(dg, Y, Ws)
    mu = api.centroids(Z.detach(), lab, rep["k"])
    params = [W.clone().requires_grad_(True) for W in Ws]
    loss = diff.SoftModLossFn.apply(diff.chain(dg, Y, params), mu, dg, 0.1)
    loss.backward()
    lo, dWo = odiff.chain_grad(g, _np(Y), [_np(W) for W in Ws], _np(mu), 0.1)
    assert abs(float(loss.detach()) - lo) <= 1e-5 * abs(lo)
    for p, ref in zip(params, dWo):
        assert rel_fro(_np(p.grad), ref) <= 1e-4


def test_weights_match_oracle(cuda):
    for layer, lin, lout in [(1, 64, 64), (2, 128, 32)]:
        W = api.gcn_weights(layer, lin, lout, 7, cuda)
        assert np.abs(_np(W) - oracle.gcn_weight(layer, lin, lout, 7)).max() <= 1e-5


def test_adam_matches_oracle(cuda):
    rng = np.random.default_rng(5)
    p0 = rng.normal(size=300)
    grads = [rng.normal(size=300) for _ in range(3)]
    p = torch.tensor(p0, dtype=torch.float32, device=cuda)
    m, v = torch.zeros_like(p), torch.zeros_like(p)
    ref = [p0.copy()]
    st = {"t": 0, "m": [np.zeros(300)], "v": [np.zeros(300)]}
    for t, gr in enumerate(grads, 1):
        api.adam_step(p, torch.tensor(gr, dtype=torch.float32, device=cuda), m, v, t, lr=0.01)
        odiff.adam(ref, [gr], st, lr=0.01)
    assert np.abs(_np(p) - ref[0]).max() <= 1e-6


def test_centroids_are_fp64_means(cuda):
    rng = np.random.default_rng(6)
    Z = rng.normal(size=(5003, 64)).astype(np.float32)
    lab = rng.integers(0, 37, size=5003)
    lab[lab == 5] = 6                       # label 5 empty: zero row
    mu = api.centroids(torch.tensor(Z, device=cuda), torch.tensor(lab, device=cuda), 37).cpu().numpy()
    for c in (0, 6, 36):
        assert np.abs(mu[c] - Z[lab == c].astype(np.float64).mean(0)).max() <= 1e-6
    assert not mu[5].any()
    with pytest.raises(api._abi.RaftgpError):
        api.centroids(torch.tensor(Z, device=cuda), torch.tensor(lab, device=cuda), 20)


def test_plan_calls_equal_one_shot_calls(cuda):
    # the same kernels on the same inputs: every output bit-identical; the loss is left on the
    # device by the plan and read back by the one-shot call, the same double either way
    g = workload("dcsbm-2k")
    dg = api.DeviceGraph.from_host(g, cuda)
    plan = api.DiffPlan(dg, 128, 80)
    rng = np.random.default_rng(5)
    for lin, lout in [(64, 32), (128, 128), (32, 64)]:
        H = torch.tensor(rng.normal(size=(g.n, lin)), dtype=torch.float32, device=cuda)
        W = torch.tensor(rng.normal(size=(lin, lout)) * 0.1, dtype=torch.float32, device=cuda)
        dHo = torch.tensor(rng.normal(size=(g.n, lout)), dtype=torch.float32, device=cuda)
        assert torch.equal(plan.layer_forward(H, W), api.gcn_layer_forward(dg, H, W))
        a, b = plan.layer_backward(H, W, dHo), api.gcn_layer_backward(dg, H, W, dHo)
        assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
        assert plan.layer_backward(H, W, dHo, need_dH=False)[0] is None
    for K, d in [(80, 64), (7, 128)]:
        Z = torch.nn.functional.normalize(torch.tensor(rng.normal(size=(g.n, d)), dtype=torch.float32, device=cuda))
        mu = Z[torch.tensor(rng.choice(g.n, K, replace=False), device=cuda)].contiguous()
        lp, dZp = plan.softmod_loss(Z, mu, 0.1)
        lo, dZo = api.softmod_loss(dg, Z, mu, 0.1)
        assert lp.device.type == "cuda" and lp.dtype == torch.float64
        assert float(lp) == lo
        assert torch.equal(dZp, dZo)


def test_plan_rejects_bad_arguments_and_graphs(cuda):
    g = workload("dcsbm-1k")
    dg = api.DeviceGraph.from_host(g, cuda)
    plan = api.DiffPlan(dg, 64, 16)
    H = torch.zeros((g.n, 128), device=cuda)
    with pytest.raises(api._abi.RaftgpError, match="wider"):
        plan.layer_forward(H, torch.zeros((128, 64), device=cuda))
    Z = torch.zeros((g.n, 64), device=cuda)
    with pytest.raises(api._abi.RaftgpError, match="larger"):
        plan.softmod_loss(Z, torch.zeros((17, 64), device=cuda), 0.1)
    with pytest.raises(api._abi.RaftgpError, match="EUNSUPPORTED"):
        api.DiffPlan(dg, 96, 16)
    bad = dg.col.clone()
    bad[17] = g.n                      # column index out of range: no plan is made
    with pytest.raises(api._abi.RaftgpError, match="EINVAL"):
        api.DiffPlan(api.DeviceGraph(g.n, dg.row_ptr, bad), 64, 16)


def test_tuning_on_a_plan_equals_one_shot_calls(cuda):
    # the loop on a plan (dL/dZ handed to the layers' backward) against autograd through the
    # one-shot calls: the same weights bit for bit, the same losses
    dg, Y, Ws, mu = _tune_setup(cuda)
    W1, l1 = diff.tune(dg, Y, Ws, mu, tau=0.1, steps=5, lr=1e-2)
    params = [W.detach().clone().requires_grad_(True) for W in Ws]
    m = [torch.zeros_like(p) for p in params]
    v = [torch.zeros_like(p) for p in params]
    l2 = []
    for t in range(1, 6):
        loss = diff.SoftModLossFn.apply(diff.chain(dg, Y, params), mu, dg, 0.1)
        for p in params:
            p.grad = None
        loss.backward()
        with torch.no_grad():
            for k, p in enumerate(params):
                api.adam_step(p.data, p.grad.contiguous(), m[k], v[k], t, 1e-2)
        l2.append(float(loss.detach()))
    assert l1 == l2
    assert all(torch.equal(a, b.detach()) for a, b in zip(W1, params))


def _tune_setup(cuda):
    g = workload("dcsbm-2k")
    dg = api.DeviceGraph.from_host(g, cuda)
    dims = (64, 64, 32)
    _, st = api.embed(dg, op="ncut", dims=dims, dtype="f32", seed=1, return_stages=True)
    Ws = [api.gcn_weights(k, dims[k - 1], dims[k], 1, cuda) for k in range(1, len(dims))]
    lab, rep = api.partition(dg, op="ncut", dims=dims, dtype="f32", kmin=2, kmax=16)
    mu = api.centroids(diff.chain(dg, st[0], Ws).detach(), lab, rep["k"])
    return dg, st[0], Ws, mu


def test_tuning_lowers_loss_and_is_deterministic(cuda):
    dg, Y, Ws, mu = _tune_setup(cuda)
    W1, l1 = diff.tune(dg, Y, Ws, mu, tau=0.1, steps=25, lr=1e-2)
    W2, l2 = diff.tune(dg, Y, Ws, mu, tau=0.1, steps=25, lr=1e-2)
    print("loss", l1[0], "->", l1[-1])
    assert l1[-1] < l1[0]
    assert l1 == l2
    assert all(torch.equal(a, b) for a, b in zip(W1, W2))


def test_tuned_weights_partition_and_score(cuda):
    out = diff.tune_partition(api.DeviceGraph.from_host(workload("dcsbm-2k"), cuda), dims=(64, 64, 32), steps=20,
                              lr=1e-2, kmax=16)
    k0, k1 = out["untrained"][1]["k"], out["tuned"][1]["k"]
    assert 2 <= k0 <= 16 and 2 <= k1 <= 16
    assert out["losses"][-1] < out["losses"][0]


def test_chain_gradient_at_full_size(cuda):
    # the differentiation form's configuration: N = 200,000, GNN 128-128-64, the untrained
    # partition's centroids; every weight gradient against the FP64 oracle
    g = workload("dcsbm-200k")
    dg = api.DeviceGraph.from_host(g, cuda)
    dims = (128, 128, 64)
    Z0, st = api.embed(dg, op="mod_full", dims=dims, dtype="f32", seed=1, return_stages=True)
    lab, rep = api.partition(dg, op="mod_full", dims=dims, dtype="f32", kmin=2, kmax=128, grid=10)
    mu = api.centroids(Z0, lab, rep["k"])
    Ws = [api.gcn_weights(k, dims[k - 1], dims[k], 1, cuda) for k in range(1, len(dims))]
    params = [W.clone().requires_grad_(True) for W in Ws]
    loss = diff.SoftModLossFn.apply(diff.chain(dg, st[0], params), mu, dg, 0.1)
    loss.backward()
    lo, dWo = odiff.chain_grad(g, _np(st[0]), [_np(W) for W in Ws], _np(mu), 0.1)
    print(f"N=200k: K*={rep['k']} loss {float(loss.detach()):.6f} (oracle {lo:.6f}); gradient rel. errors "
          + ", ".join(f"{rel_fro(_np(p.grad), r):.2e}" for p, r in zip(params, dWo)))
    assert abs(float(loss.detach()) - lo) <= 1e-5 * abs(lo)
    for p, ref in zip(params, dWo):
        assert rel_fro(_np(p.grad), ref) <= 1e-4
