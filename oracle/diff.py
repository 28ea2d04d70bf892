"""FP64 oracle for the differentiation form -- TEST INFRASTRUCTURE ONLY.

The GNN weights of the Eq. 6 chain may be tuned against a relaxed (soft-assignment)
modularity.  The paper trains nothing (its GNN is random, Section III-B); the loss below is
a build choice, written down here in plain NumPy FP64 with the gradient derived by hand:

  layer k:   P = H W_k,  A = Ahat P,  T = tanh(A),  H' = T / ||T||_row   (a zero row stays 0)
             Ahat = Dhat^-1/2 (A + I) Dhat^-1/2, dhat = d + 1                        (Eq. 6)
  soft assignment against fixed centroids mu (K x d), temperature tau:
             D_ic = ||z_i - mu_c||^2,   S_i = softmax_c(-D_ic / tau)
  loss       L = -(1 / 2e) [ tr(S^T A S) - ||d^T S||^2 / 2e ]
             (with a one-hot S this is -Mod of the partition, Eq. 3; with a uniform S it is 0)

Backward, in the order it is evaluated:
  dL/dS     = -(1/e) [ A S - d (d^T S) / 2e ]                          (A symmetric)
  dL/dlogit = S * (dL/dS - rowsum(S * dL/dS)),   logit = -D / tau
  dL/dD     = -(1/tau) dL/dlogit
  dL/dz_i   = sum_c dL/dD_ic * 2 (z_i - mu_c)
  layer:    dT = (dH' - H' rowsum(H' * dH')) / ||T||_row,   dA = dT * (1 - T^2),
            dP = Ahat dA (Ahat symmetric),   dW_k = H^T dP,   dH = dP W_k^T

Only the tests may import this module; the library never does.  It shares no code with the
CUDA library (the layer forward is cross-checked against the C oracle's Eq. 6 layer).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def _adjacency(g):
    n = g.n
    rp = np.asarray(g.row_ptr, dtype=np.int64)
    col = np.asarray(g.col, dtype=np.int64)
    return sp.csr_matrix((np.ones(col.shape[0]), col, rp), shape=(n, n))


def degrees(g):
    return np.diff(np.asarray(g.row_ptr, dtype=np.int64)).astype(np.float64)


def a_hat(g):
    """Dhat^-1/2 (A + I) Dhat^-1/2 with dhat = d + 1 (Eq. 6)."""
    A = _adjacency(g)
    s = 1.0 / np.sqrt(degrees(g) + 1.0)
    S = sp.diags(s)
    return (S @ (A + sp.identity(g.n, format="csr")) @ S).tocsr()


def layer_forward(Ah, H, W):
    """One Eq. 6 layer: returns (H_out, T, r) with T = tanh(Ahat H W), r = row norms of T."""
    T = np.tanh(Ah @ (H @ W))
    r = np.sqrt((T * T).sum(axis=1))
    Hout = np.where(r[:, None] > 0, T / np.where(r > 0, r, 1.0)[:, None], 0.0)
    return Hout, T, r


def layer_backward(Ah, H, W, T, r, Hout, dHout):
    """Gradients of one layer: returns (dH_in, dW)."""
    safe = np.where(r > 0, r, 1.0)[:, None]
    dT = np.where(r[:, None] > 0, (dHout - Hout * (Hout * dHout).sum(axis=1, keepdims=True)) / safe, 0.0)
    dA = dT * (1.0 - T * T)
    dP = Ah @ dA
    return dP @ W.T, H.T @ dP


def soft_assignment(Z, mu, tau):
    # direct-form squared distances, computed in row blocks to bound the temporary
    D = np.empty((Z.shape[0], mu.shape[0]))
    for r0 in range(0, Z.shape[0], 2048):
        D[r0:r0 + 2048] = ((Z[r0:r0 + 2048, None, :] - mu[None, :, :]) ** 2).sum(axis=2)
    logit = -D / tau
    logit -= logit.max(axis=1, keepdims=True)
    E = np.exp(logit)
    return E / E.sum(axis=1, keepdims=True), D


def softmod_loss(g, Z, mu, tau):
    A = _adjacency(g)
    d = degrees(g)
    two_e = d.sum()
    S, _ = soft_assignment(Z, mu, tau)
    dS = d @ S
    return -(np.sum(S * (A @ S)) - dS @ dS / two_e) / two_e


def softmod_grad(g, Z, mu, tau):
    """(loss, dL/dZ)."""
    A = _adjacency(g)
    d = degrees(g)
    two_e = d.sum()
    S, _ = soft_assignment(Z, mu, tau)
    AS = A @ S
    dTS = d @ S
    loss = -(np.sum(S * AS) - dTS @ dTS / two_e) / two_e
    gS = -(AS - np.outer(d, dTS) / two_e) / (two_e / 2.0)
    gl = S * (gS - (S * gS).sum(axis=1, keepdims=True))
    G = -gl / tau
    dZ = 2.0 * (G.sum(axis=1)[:, None] * Z - G @ mu)
    return loss, dZ


def chain_forward(g, Y, Ws):
    """Every layer's output [H_0 = Y, H_1, ..., H_L]."""
    Ah = a_hat(g)
    Hs = [np.asarray(Y, dtype=np.float64)]
    for W in Ws:
        Hs.append(layer_forward(Ah, Hs[-1], np.asarray(W, dtype=np.float64))[0])
    return Hs


def chain_loss(g, Y, Ws, mu, tau):
    return softmod_loss(g, chain_forward(g, Y, Ws)[-1], mu, tau)


def chain_grad(g, Y, Ws, mu, tau):
    """(loss, [dL/dW_1, ..., dL/dW_L]) through the whole chain."""
    Ah = a_hat(g)
    Ws = [np.asarray(W, dtype=np.float64) for W in Ws]
    Hs = [np.asarray(Y, dtype=np.float64)]
    saved = []
    for W in Ws:
        Hout, T, r = layer_forward(Ah, Hs[-1], W)
        saved.append((T, r, Hout))
        Hs.append(Hout)
    loss, dH = softmod_grad(g, Hs[-1], mu, tau)
    dWs = [None] * len(Ws)
    for k in range(len(Ws) - 1, -1, -1):
        T, r, Hout = saved[k]
        dH, dWs[k] = layer_backward(Ah, Hs[k], Ws[k], T, r, Hout, dH)
    return loss, dWs


def adam(params, grads, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma and Ba, 2015) in place; state = dict(t, m, v)."""
    state["t"] += 1
    t = state["t"]
    for k, (p, gr) in enumerate(zip(params, grads)):
        state["m"][k] = b1 * state["m"][k] + (1 - b1) * gr
        state["v"][k] = b2 * state["v"][k] + (1 - b2) * gr * gr
        mh = state["m"][k] / (1 - b1 ** t)
        vh = state["v"][k] / (1 - b2 ** t)
        p -= lr * mh / (np.sqrt(vh) + eps)
