"""Pins of the differentiation oracle (oracle/diff.py): its hand-derived gradient against
central finite differences in FP64, its loss against Eq. 3 modularity (the one-hot limit) and
against the uniform-assignment closed form (0), its layer against the C oracle's Eq. 6 layer."""
import numpy as np
import pytest

import oracle
from oracle import diff
from inputs.small import random_graph, ring_of_cliques


def _setup(seed=0, n=40, dims=(6, 5, 4), K=3):
    rng = np.random.default_rng(seed)
    g = random_graph(n, 0.15, seed, isolated=2)
    Y = rng.normal(size=(n, dims[0]))
    Ws = [rng.normal(size=(dims[k], dims[k + 1])) * np.sqrt(2.0 / (dims[k] + dims[k + 1]))
          for k in range(len(dims) - 1)]
    mu = rng.normal(size=(K, dims[-1]))
    mu /= np.linalg.norm(mu, axis=1, keepdims=True)
    return g, Y, Ws, mu


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_chain_gradient_matches_central_differences():
    g, Y, Ws, mu = _setup()
    tau, h = 0.3, 1e-6
    loss, dWs = diff.chain_grad(g, Y, Ws, mu, tau)
    assert np.isclose(loss, diff.chain_loss(g, Y, Ws, mu, tau), rtol=0, atol=1e-15)
    for k, W in enumerate(Ws):
        fd = np.zeros_like(W)
        for idx in np.ndindex(W.shape):
            Wp = [w.copy() for w in Ws]
            Wm = [w.copy() for w in Ws]
            Wp[k][idx] += h
            Wm[k][idx] -= h
            fd[idx] = (diff.chain_loss(g, Y, Wp, mu, tau) - diff.chain_loss(g, Y, Wm, mu, tau)) / (2 * h)
        assert _rel(dWs[k], fd) <= 1e-6, k


def test_loss_gradient_in_z_matches_central_differences():
    g, Y, Ws, mu = _setup(seed=1)
    Z = diff.chain_forward(g, Y, Ws)[-1]
    tau, h = 0.2, 1e-6
    _, dZ = diff.softmod_grad(g, Z, mu, tau)
    fd = np.zeros_like(Z)
    for idx in np.ndindex(Z.shape):
        Zp, Zm = Z.copy(), Z.copy()
        Zp[idx] += h
        Zm[idx] -= h
        fd[idx] = (diff.softmod_loss(g, Zp, mu, tau) - diff.softmod_loss(g, Zm, mu, tau)) / (2 * h)
    assert _rel(dZ, fd) <= 1e-6


def test_one_hot_limit_is_minus_modularity():
    # ring of 5 cliques of 6; points placed at their clique's centroid plus small noise, so
    # the nearest centroid is the clique and a tiny temperature makes S one-hot
    g = ring_of_cliques(5, 6)
    rng = np.random.default_rng(3)
    mu = np.eye(5, 8)
    labels = np.arange(g.n) // 6
    Z = mu[labels] + 0.01 * rng.normal(size=(g.n, 8))
    loss = diff.softmod_loss(g, Z, mu, 1e-4)
    _, _, mod, _ = oracle.score(g, labels, 5)
    assert abs(loss + mod) <= 1e-12


def test_uniform_assignment_gives_zero():
    g, Y, Ws, mu = _setup(seed=2)
    Z = diff.chain_forward(g, Y, Ws)[-1]
    assert abs(diff.softmod_loss(g, Z, mu, 1e9)) <= 1e-9


@pytest.mark.parametrize("isolated", [0, 3])
def test_layer_forward_matches_c_oracle(isolated):
    rng = np.random.default_rng(4)
    g = random_graph(50, 0.1, 4, isolated=isolated)
    H = rng.normal(size=(g.n, 8))
    W = rng.normal(size=(8, 6))
    mine = diff.layer_forward(diff.a_hat(g), H, W)[0]
    assert np.abs(mine - oracle.gcn_layer(g, H, W)).max() <= 1e-12


def test_adam_first_step_moves_by_lr_times_sign():
    p = [np.array([1.0, -2.0, 3.0])]
    st = {"t": 0, "m": [np.zeros(3)], "v": [np.zeros(3)]}
    diff.adam(p, [np.array([0.5, -4.0, 0.0])], st, lr=0.1)
    # after one step m_hat = g and v_hat = g^2, so the move is lr * g / (|g| + eps)
    assert np.allclose(p[0], [0.9, -1.9, 3.0], atol=1e-7)
