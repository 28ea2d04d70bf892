"""Algorithm 2 on the GPU: the drawn edge lists equal the FP64 oracle's edge for edge (same
Philox draws, same prefix-mass formulas, same order), including empty and one-node blocks,
pairs with Omega = 0 and tables of many segments; the device CSR build equals the sorted
CSR built on the host; malformed parameters are rejected; at 1M nodes the edge count lies
within the bounds the model gives."""
import numpy as np
import pytest
import torch

import oracle
from inputs.dcsbm import WORKLOADS, dcsbm_params, from_edges
from paper_2312_01560_gb300 import api

pytestmark = pytest.mark.gpu


def _gpu(block, theta, om, seed, cuda):
    s, d, w = api.sbm_sample(torch.as_tensor(block, device=cuda), torch.as_tensor(theta, device=cuda),
                             torch.as_tensor(om, device=cuda), seed=seed, weights=True)
    torch.cuda.synchronize()
    return s.cpu().numpy(), d.cpu().numpy(), w.cpu().numpy()


def _handmade():
    rng = np.random.default_rng(9)
    n, K = 500, 6
    block = rng.integers(0, 3, n).astype(np.int32)
    block[17] = 4                                  # a one-node block; block 3 stays empty
    block[[5, 99, 250]] = 5
    theta = rng.uniform(0.1, 4.0, n)
    theta[40] = 0.0                                # a node that can have no edge
    om = rng.uniform(0.0, 0.02, (K, K))
    om = (om + om.T) / 2
    om[0, 2] = om[2, 0] = 0.0                      # a pair with no edge
    om[5, 5] = 3.0
    return block, theta, om


@pytest.mark.parametrize("case", ["handmade", "dcsbm-50k", "dcsbm-2k"])
def test_edges_equal_the_oracle(cuda, case):
    if case == "handmade":
        block, theta, om = _handmade()
    else:
        block, theta, om = dcsbm_params(seed=3, **WORKLOADS[case])
    for seed in (1, 2):
        s, d, w = _gpu(block, theta, om, seed, cuda)
        so, do, wo = oracle.sbm_sample(block, theta, om, seed)
        print(f"{case} seed {seed}: {len(s)} edges (oracle {len(so)})")
        assert len(s) == len(so)
        assert np.array_equal(s, so) and np.array_equal(d, do) and np.array_equal(w, wo)


def test_csr_build_equals_the_host_csr(cuda):
    block, theta, om = dcsbm_params(seed=4, **WORKLOADS["dcsbm-50k"])
    s, d, _ = _gpu(block, theta, om, 5, cuda)
    g = api.coo_to_csr(len(block), torch.as_tensor(s, device=cuda), torch.as_tensor(d, device=cuda))
    torch.cuda.synchronize()
    ref = from_edges(len(block), s.astype(np.int64), d.astype(np.int64))
    assert np.array_equal(g.row_ptr.cpu().numpy(), ref.row_ptr)
    assert np.array_equal(g.col.cpu().numpy(), ref.col)
    # a hub longer than one warp's sort (block path) and isolated nodes
    n = 3000
    hub_v = np.arange(1, 2001)
    u = np.concatenate([np.zeros(2000, np.int64), np.arange(100, 600)])
    v = np.concatenate([hub_v, np.arange(1100, 1600)])
    g = api.coo_to_csr(n, torch.as_tensor(u, device=cuda), torch.as_tensor(v, device=cuda))
    ref = from_edges(n, u, v)
    assert np.array_equal(g.row_ptr.cpu().numpy(), ref.row_ptr) and np.array_equal(g.col.cpu().numpy(), ref.col)


def test_bad_parameters_are_rejected(cuda):
    block, theta, om = _handmade()
    bad = block.copy()
    bad[3] = om.shape[0]
    with pytest.raises(api._abi.RaftgpError, match="EINVAL"):
        _gpu(bad, theta, om, 1, cuda)
    th = theta.copy()
    th[7] = -1.0
    with pytest.raises(api._abi.RaftgpError, match="EINVAL"):
        _gpu(block, th, om, 1, cuda)
    o2 = om.copy()
    o2[1, 2] = np.nan
    with pytest.raises(api._abi.RaftgpError, match="EINVAL"):
        _gpu(block, theta, o2, 1, cuda)
    u = torch.tensor([0, 1, 2], dtype=torch.int32, device=cuda)
    with pytest.raises(api._abi.RaftgpError, match="EINVAL"):
        api.coo_to_csr(5, u, torch.tensor([1, 1, 3], dtype=torch.int32, device=cuda))   # a self loop
    with pytest.raises(api._abi.RaftgpError, match="EINVAL"):
        api.coo_to_csr(5, u, torch.tensor([1, 2, 9], dtype=torch.int32, device=cuda))   # outside [0, n)
    star = torch.arange(1, 20001, dtype=torch.int32, device=cuda)
    with pytest.raises(api._abi.RaftgpError, match="EUNSUPPORTED"):
        api.coo_to_csr(20001, torch.zeros_like(star), star)                             # a row of 20,000


def test_emit_checks_the_count(cuda):
    import ctypes as C
    block, theta, om = _handmade()
    bt, tt, ot = (torch.as_tensor(x, device=cuda) for x in (block, theta.astype(np.float64), om))
    p = api._abi.Sbm()
    p.n, p.k, p.seed = len(block), om.shape[0], 1
    p.block, p.theta, p.omega = bt.data_ptr(), tt.data_ptr(), ot.data_ptr()
    ws = torch.empty(int(api.lib().raftgp_sbm_workspace_size(p.n, p.k)), dtype=torch.uint8, device=cuda)
    m = C.c_int64(0)
    api.check(api.lib().raftgp_sbm_count(C.byref(p), C.byref(m), C.c_void_p(ws.data_ptr()), ws.numel(), None))
    out = torch.empty(m.value + 8, dtype=torch.int32, device=cuda)
    st = api.lib().raftgp_sbm_emit(C.byref(p), C.c_void_p(out.data_ptr()), C.c_void_p(out.data_ptr()), None,
                                   m.value + 1, C.c_void_p(ws.data_ptr()), ws.numel(), None)
    assert st == api._abi.EINVAL


def test_million_node_graph_size(cuda):
    """dcsbm-1m parameters: the edge count lies between the model's bounds sum(lambda -
    lambda^2 / 2) and sum(lambda) (5 standard deviations of slack), the mean degree is near
    its target and two draws with one seed are identical."""
    cfg = WORKLOADS["dcsbm-1m"]
    block, theta, om = dcsbm_params(seed=0, **cfg)
    s, d, _ = _gpu(block, theta, om, 7, cuda)
    s2, d2, _ = _gpu(block, theta, om, 7, cuda)
    assert np.array_equal(s, s2) and np.array_equal(d, d2)
    K = om.shape[0]
    t1 = np.bincount(block, weights=theta, minlength=K)
    t2 = np.bincount(block, weights=theta ** 2, minlength=K)
    t4 = np.bincount(block, weights=theta ** 4, minlength=K)
    a_in = np.diag(om)
    # sum over i < j of lambda and lambda^2, within blocks and between blocks
    lam1 = np.sum(a_in * (t1 ** 2 - t2) / 2) + om[0, 1] * (t1.sum() ** 2 - np.sum(t1 ** 2)) / 2
    lam2 = np.sum(a_in ** 2 * (t2 ** 2 - t4) / 2) + om[0, 1] ** 2 * (t2.sum() ** 2 - np.sum(t2 ** 2)) / 2
    m = len(s)
    sd = np.sqrt(lam1)
    print(f"1M nodes: {m} edges, bounds [{lam1 - lam2 / 2:.0f}, {lam1:.0f}], mean degree {2 * m / len(block):.2f}")
    assert lam1 - lam2 / 2 - 5 * sd <= m <= lam1 + 5 * sd
    assert (s != d).all()
    assert abs(2 * m / len(block) - cfg["mean_degree"]) < 0.1 * cfg["mean_degree"]
