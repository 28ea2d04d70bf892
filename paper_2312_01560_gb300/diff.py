"""The differentiation form: Eq. 6 layers and the relaxed soft-assignment modularity as
torch.autograd.Functions whose forward and backward are the library's hand-written kernels,
and a tuning loop (Adam, in the library) for the GNN weights.

The paper keeps its GNN random (Section III-B); tuning is an optional extra.  Only the layer
inputs are kept for the backward: each layer's pre-activation is computed again there."""
from __future__ import annotations

import torch

from . import api


def _forward(g, H, W):
    return g.layer_forward(H, W) if isinstance(g, api.DiffPlan) else api.gcn_layer_forward(g, H, W)


def _backward(g, H, W, dH_out, need_dH):
    if isinstance(g, api.DiffPlan):
        return g.layer_backward(H, W, dH_out, need_dH=need_dH)
    return api.gcn_layer_backward(g, H, W, dH_out, need_dH=need_dH)


class GCNLayerFn(torch.autograd.Function):
    """H_out = rownorm(tanh(Ahat (H W))) (Eq. 6).  `g` is a DeviceGraph (each call checks it)
    or an api.DiffPlan (checked once)."""

    @staticmethod
    def forward(ctx, H, W, g):
        ctx.g = g
        ctx.save_for_backward(H, W)
        return _forward(g, H.contiguous(), W.contiguous())

    @staticmethod
    def backward(ctx, dH_out):
        H, W = ctx.saved_tensors
        dH, dW = _backward(ctx.g, H.contiguous(), W.contiguous(), dH_out.contiguous(), ctx.needs_input_grad[0])
        return dH, dW, None


class SoftModLossFn(torch.autograd.Function):
    """-(tr(S^T A S) - ||d^T S||^2 / 2e) / 2e with S = softmax(-||z - mu||^2 / tau).  With a
    DeviceGraph the loss is a host float64 tensor (the call synchronises); with an
    api.DiffPlan it stays on the device."""

    @staticmethod
    def forward(ctx, Z, mu, g, tau):
        if isinstance(g, api.DiffPlan):
            loss, dZ = g.softmod_loss(Z.contiguous(), mu.contiguous(), tau, need_grad=True)
        else:
            value, dZ = api.softmod_loss(g, Z.contiguous(), mu.contiguous(), tau, need_grad=True)
            loss = torch.tensor(value, dtype=torch.float64)
        ctx.save_for_backward(dZ)
        return loss

    @staticmethod
    def backward(ctx, grad_loss):
        (dZ,) = ctx.saved_tensors
        if grad_loss.device.type == "cpu":
            scale = float(grad_loss)
            return (dZ if scale == 1.0 else dZ * scale), None, None, None
        return dZ * grad_loss.to(dZ.dtype), None, None, None


def chain(g, Y, Ws):
    H = Y
    for W in Ws:
        H = GCNLayerFn.apply(H, W, g)
    return H


def tune(g, Y, Ws, mu, tau=0.1, steps=200, lr=1e-3, betas=(0.9, 0.999), eps=1e-8, plan=None):
    """Adam on the GNN weights against the relaxed modularity of the final layer.
    Returns (tuned weights, loss before each step).

    The steps run on an api.DiffPlan (made here unless given), so nothing synchronises
    inside the loop: dL/dZ from the loss call is passed straight into the layers' backward,
    and the losses are read back once, at the end."""
    params = [W.detach().clone().contiguous().requires_grad_(True) for W in Ws]
    if plan is None:
        width = max(max(W.shape) for W in Ws)
        plan = api.DiffPlan(g, width, mu.shape[0])
    m = [torch.zeros_like(p) for p in params]
    v = [torch.zeros_like(p) for p in params]
    losses = []
    for t in range(1, steps + 1):
        Z = chain(plan, Y, params)
        loss, dZ = plan.softmod_loss(Z.detach(), mu.contiguous(), tau)
        for p in params:
            p.grad = None
        Z.backward(dZ)
        with torch.no_grad():
            for k, p in enumerate(params):
                api.adam_step(p.data, p.grad.contiguous(), m[k], v[k], t, lr, betas[0], betas[1], eps)
        losses.append(loss)
    losses = torch.stack(losses).cpu().tolist() if losses else []
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
