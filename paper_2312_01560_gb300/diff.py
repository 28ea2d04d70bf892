"""The differentiation form: Eq. 6 layers and the relaxed soft-assignment modularity as
torch.autograd.Functions whose forward and backward are the library's hand-written kernels,
and a tuning loop (Adam, in the library) for the GNN weights.

The paper keeps its GNN random (Section III-B); tuning is an optional extra.  Only the layer
inputs are kept for the backward: each layer's pre-activation is computed again there."""
from __future__ import annotations

import torch

from . import api


class GCNLayerFn(torch.autograd.Function):
    """H_out = rownorm(tanh(Ahat (H W))) (Eq. 6)."""

    @staticmethod
    def forward(ctx, H, W, g):
        ctx.g = g
        ctx.save_for_backward(H, W)
        return api.gcn_layer_forward(g, H.contiguous(), W.contiguous())

    @staticmethod
    def backward(ctx, dH_out):
        H, W = ctx.saved_tensors
        dH, dW = api.gcn_layer_backward(ctx.g, H.contiguous(), W.contiguous(), dH_out.contiguous(),
                                        need_dH=ctx.needs_input_grad[0])
        return dH, dW, None


class SoftModLossFn(torch.autograd.Function):
    """-(tr(S^T A S) - ||d^T S||^2 / 2e) / 2e with S = softmax(-||z - mu||^2 / tau)."""

    @staticmethod
    def forward(ctx, Z, mu, g, tau):
        loss, dZ = api.softmod_loss(g, Z.contiguous(), mu.contiguous(), tau, need_grad=True)
        ctx.save_for_backward(dZ)
        return torch.tensor(loss, dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad_loss):
        (dZ,) = ctx.saved_tensors
        scale = float(grad_loss)
        return (dZ if scale == 1.0 else dZ * scale), None, None, None


def chain(g, Y, Ws):
    H = Y
    for W in Ws:
        H = GCNLayerFn.apply(H, W, g)
    return H


def tune(g, Y, Ws, mu, tau=0.1, steps=200, lr=1e-3, betas=(0.9, 0.999), eps=1e-8):
    """Adam on the GNN weights against the relaxed modularity of the final layer.
    Returns (tuned weights, loss before each step)."""
    params = [W.detach().clone().contiguous().requires_grad_(True) for W in Ws]
    m = [torch.zeros_like(p) for p in params]
    v = [torch.zeros_like(p) for p in params]
    losses = []
    for t in range(1, steps + 1):
        loss = SoftModLossFn.apply(chain(g, Y, params), mu, g, tau)
        for p in params:
            p.grad = None
        loss.backward()
        with torch.no_grad():
            for k, p in enumerate(params):
                api.adam_step(p.data, p.grad.contiguous(), m[k], v[k], t, lr, betas[0], betas[1], eps)
        losses.append(float(loss.detach()))
    return [p.detach() for p in params], losses


def tune_partition(g, op="ncut", dims=(128, 128, 64), tau=0.1, steps=200, lr=1e-3, kmin=2, kmax=None, grid=10,
                   seed=1):
    """The whole differentiation form on one graph:
    1. the untrained FP32 partition (projection, random GNN, model selection) gives K* and
       the centroids mu of its labels;
    2. the GNN weights, starting from the ones the embedding drew, are tuned for `steps` Adam
       steps against the relaxed modularity with mu fixed;
    3. the graph is partitioned again with the tuned weights.
    Returns a dict with both partitions, the losses and the tuned weights."""
    kmax = kmax or min(128, g.n)
    lab0, rep0 = api.partition(g, op=op, dims=dims, dtype="f32", kmin=kmin, kmax=kmax, grid=grid, embed_seed=seed)
    Z0, st = api.embed(g, op=op, dims=dims, dtype="f32", seed=seed, return_stages=True)
    mu = api.centroids(Z0, lab0, rep0["k"])
    Y = st[0]
    Ws = [api.gcn_weights(k, dims[k - 1], dims[k], seed, Y.device) for k in range(1, len(dims))]
    Wt, losses = tune(g, Y, Ws, mu, tau=tau, steps=steps, lr=lr)
    lab1, rep1 = api.partition(g, op=op, dims=dims, dtype="f32", kmin=kmin, kmax=kmax, grid=grid, embed_seed=seed,
                               W=Wt)
    return {"untrained": (lab0, rep0), "tuned": (lab1, rep1), "losses": losses, "W": Wt, "mu": mu}
