"""Python binding of the RaftGP CUDA library: torch tensors in, torch tensors out.

Argument marshalling only -- every step runs in libraftgp.so's kernels.  PyTorch provides
device memory and the stream; the workspace is a cached device byte tensor.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field

import torch

from . import _abi
from ._abi import check, lib


@dataclass
class DeviceGraph:
    """A symmetric CSR graph resident on the GPU."""
    n: int
    row_ptr: torch.Tensor   # int32 or int64, n+1
    col: torch.Tensor       # int32, nnz

    @property
    def nnz(self) -> int:
        return int(self.col.numel())

    @property
    def n_edges(self) -> int:
        return self.nnz // 2

    @classmethod
    def from_host(cls, g, device="cuda", row_ptr_bits=None):
        """From any object with n, row_ptr and col numpy arrays (e.g. inputs.dcsbm.Graph)."""
        import numpy as np
        rp = np.asarray(g.row_ptr)
        bits = row_ptr_bits or (32 if rp[-1] < 2 ** 31 - 1 else 64)
        rp_t = torch.from_numpy(rp.astype(np.int32 if bits == 32 else np.int64)).to(device)
        col_t = torch.from_numpy(np.asarray(g.col, dtype=np.int32)).to(device)
        return cls(int(g.n), rp_t, col_t)

    def csr(self) -> _abi.Csr:
        bits = 32 if self.row_ptr.dtype == torch.int32 else 64
        return _abi.Csr(self.n, self.nnz, self.row_ptr.data_ptr(), bits, self.col.data_ptr() if self.nnz else None)


_ws = {}


def _workspace(nbytes: int, device) -> torch.Tensor:
    key = str(device)
    t = _ws.get(key)
    if t is None or t.numel() < nbytes:
        t = torch.empty(max(nbytes, 1 << 20), dtype=torch.uint8, device=device)
        _ws[key] = t
    return t


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dtype_code(dtype) -> int:
    return _abi.DTYPE[dtype] if isinstance(dtype, str) else int(dtype)


def _torch_dtype(code: int):
    return torch.bfloat16 if code == 1 else torch.float32


def embed_opts(op="ncut", dims=(64, 64, 32), dtype="f32", seed=1, theta=None, W=None, stages=None):
    o = _abi.EmbedOpts()
    o.op = _abi.OP[op] if isinstance(op, str) else int(op)
    o.n_layers = len(dims) - 1
    for k, v in enumerate(dims):
        o.dims[k] = int(v)
    o.dtype = _dtype_code(dtype)
    o.seed = int(seed)
    o.theta = theta.data_ptr() if theta is not None else None
    if W is not None:
        for k, w in enumerate(W):
            o.W[k] = w.data_ptr()
    if stages is not None:
        for k, t in enumerate(stages):
            o.stage_out[k] = t.data_ptr() if t is not None else None
    return o


def _code(table, v):
    return table[v] if isinstance(v, str) else int(v)


def select_opts(kmin=2, kmax=40, grid=0, iters=50, criterion="mod", assign="ffma", batch=0, seed=2, recheck="fp32"):
    o = _abi.SelectOpts()
    o.kmin, o.kmax, o.grid, o.iters = int(kmin), int(kmax), int(grid), int(iters)
    o.criterion = _code(_abi.CRIT, criterion)
    o.assign = _code(_abi.ASSIGN, assign)
    o.batch = int(batch)
    o.recheck = _code(_abi.RECHECK, recheck)
    o.seed = int(seed)
    return o


def workspace_size(g: DeviceGraph, eopts=None, sopts=None, d=0) -> int:
    csr = g.csr()
    return lib().raftgp_workspace_size(C.byref(csr), C.byref(eopts) if eopts is not None else None,
                                       C.byref(sopts) if sopts is not None else None, int(d))


def embed(g: DeviceGraph, op="ncut", dims=(64, 64, 32), dtype="f32", seed=1, theta=None, W=None,
          return_stages=False, stream=None):
    """Stages 1-2 (Eq. 5 projection and the Eq. 6 GCN): returns Z (N x dims[-1])."""
    code = _dtype_code(dtype)
    dev = g.col.device
    Z = torch.empty((g.n, dims[-1]), dtype=_torch_dtype(code), device=dev)
    stages = [torch.empty((g.n, w), dtype=_torch_dtype(code), device=dev) for w in dims] if return_stages else None
    if theta is not None:
        theta = theta.to(dev, torch.float32).contiguous()
    if W is not None:
        W = [w.to(dev, torch.float32).contiguous() for w in W]
    o = embed_opts(op, dims, code, seed, theta, W, stages)
    csr = g.csr()
    nbytes = lib().raftgp_workspace_size(C.byref(csr), C.byref(o), None, 0)
    ws = _workspace(nbytes, dev)
    check(lib().raftgp_embed(C.byref(csr), C.byref(o), C.c_void_p(Z.data_ptr()), C.c_void_p(ws.data_ptr()),
                             ws.numel(), _stream(stream)))
    return (Z, stages) if return_stages else Z


def _result(cap):
    r = _abi.SelectResult()
    keep = ((C.c_int32 * cap)(), (C.c_double * cap)(), (C.c_double * cap)(), (C.c_int32 * cap)())
    r.cand_cap = cap
    r.cand_k, r.cand_mod, r.cand_ncut, r.cand_passes = (C.cast(keep[0], C.POINTER(C.c_int32)),
                                                        C.cast(keep[1], C.POINTER(C.c_double)),
                                                        C.cast(keep[2], C.POINTER(C.c_double)),
                                                        C.cast(keep[3], C.POINTER(C.c_int32)))
    return r, keep


def _unpack(r, keep):
    n = r.n_cand
    return {"k": r.k_best,
            "cands": [(keep[0][i], keep[1][i], keep[2][i], keep[3][i]) for i in range(min(n, r.cand_cap))]}


def select(g: DeviceGraph, Z: torch.Tensor, kmin=2, kmax=40, grid=0, iters=50, criterion="mod", assign="ffma",
           batch=0, seed=2, stream=None, labels=None, recheck="fp32"):
    """Stage 3: returns (labels int32[N] on the device, report dict)."""
    code = 1 if Z.dtype == torch.bfloat16 else 0
    o = select_opts(kmin, kmax, grid, iters, criterion, assign, batch, seed, recheck)
    csr = g.csr()
    d = Z.shape[1]
    nbytes = lib().raftgp_workspace_size(C.byref(csr), None, C.byref(o), d)
    ws = _workspace(nbytes, Z.device)
    if labels is None:
        labels = torch.empty(g.n, dtype=torch.int32, device=Z.device)
    r, keep = _result((kmax - kmin + 1) + 2 * grid + 2)
    Zc = Z.contiguous()
    check(lib().raftgp_select(C.byref(csr), C.c_void_p(Zc.data_ptr()), d, code, C.byref(o),
                              C.c_void_p(labels.data_ptr()), C.byref(r), C.c_void_p(ws.data_ptr()), ws.numel(),
                              _stream(stream)))
    return labels, _unpack(r, keep)


def partition(g: DeviceGraph, op="ncut", dims=(64, 64, 32), dtype="f32", embed_seed=1, kmin=2, kmax=40, grid=0,
              iters=50, criterion="mod", assign="ffma", batch=0, select_seed=2, stream=None, labels=None, W=None,
              recheck="fp32"):
    """Stages 1-3 end to end: returns (labels, report).  W: optional GNN weights (FP32)."""
    if W is not None:
        W = [w.to(g.col.device, torch.float32).contiguous() for w in W]
    eo = embed_opts(op, dims, dtype, embed_seed, None, W)
    so = select_opts(kmin, kmax, grid, iters, criterion, assign, batch, select_seed, recheck)
    csr = g.csr()
    nbytes = lib().raftgp_workspace_size(C.byref(csr), C.byref(eo), C.byref(so), 0)
    ws = _workspace(nbytes, g.col.device)
    if labels is None:
        labels = torch.empty(g.n, dtype=torch.int32, device=g.col.device)
    r, keep = _result((kmax - kmin + 1) + 2 * grid + 2)
    check(lib().raftgp_partition(C.byref(csr), C.byref(eo), C.byref(so), C.c_void_p(labels.data_ptr()), C.byref(r),
                                 C.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream)))
    return labels, _unpack(r, keep)


def score(g: DeviceGraph, labels: torch.Tensor, K: int, stream=None):
    """Eq. 3 / Eq. 1 of a given partition: returns (m, vol, mod, ncut)."""
    dev = g.col.device
    m = torch.empty(K, dtype=torch.int64, device=dev)
    vol = torch.empty(K, dtype=torch.int64, device=dev)
    mod = C.c_double(0)
    ncut = C.c_double(0)
    ws = _workspace(4096 + 16 * g.n + 4096, dev)
    csr = g.csr()
    lab = labels.to(dev, torch.int32).contiguous()
    check(lib().raftgp_score(C.byref(csr), C.c_void_p(lab.data_ptr()), int(K), C.c_void_p(m.data_ptr()),
                             C.c_void_p(vol.data_ptr()), C.byref(mod), C.byref(ncut), C.c_void_p(ws.data_ptr()),
                             ws.numel(), _stream(stream)))
    return m, vol, mod.value, ncut.value


def debug_seed_skip_block(block: int):
    """Test hook: block `block` of the persistent seeding kernel leaves at round 2 without
    arriving at the grid barrier (the bounded wait of the others runs out); -1 turns it off."""
    lib().raftgp_debug_seed_skip_block(int(block))


def kmeanspp(Z: torch.Tensor, K: int, seed: int, stream=None):
    n, d = Z.shape
    code = 1 if Z.dtype == torch.bfloat16 else 0
    seeds = torch.empty(K, dtype=torch.int32, device=Z.device)
    ws = _workspace(7 * n + 8 * max(n // 1024 + 1, 2048) + 4 * K + 4096, Z.device)
    Zc = Z.contiguous()
    check(lib().raftgp_kmeanspp(C.c_void_p(Zc.data_ptr()), n, d, code, int(K), int(seed),
                                C.c_void_p(seeds.data_ptr()), C.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream)))
    return seeds


def lloyd(Z: torch.Tensor, mu0: torch.Tensor, iters=50, assign="ffma", recheck="fp32", stream=None):
    """Lloyd's iterations from mu0: returns (labels int32[N], mu float32[K, d], passes)."""
    n, d = Z.shape
    K = mu0.shape[0]
    code = 1 if Z.dtype == torch.bfloat16 else 0
    labels = torch.empty(n, dtype=torch.int32, device=Z.device)
    mu = torch.empty((K, d), dtype=torch.float32, device=Z.device)
    m0 = mu0.to(Z.device, torch.float32).contiguous()
    ws = _workspace(int(lib().raftgp_lloyd_workspace_size(n, d, int(K))), Z.device)
    passes = C.c_int32(0)
    Zc = Z.contiguous()
    check(lib().raftgp_lloyd(C.c_void_p(Zc.data_ptr()), n, d, code, C.c_void_p(m0.data_ptr()), int(K),
                             int(iters), _code(_abi.ASSIGN, assign), _code(_abi.RECHECK, recheck),
                             C.c_void_p(labels.data_ptr()), C.c_void_p(mu.data_ptr()), C.byref(passes),
                             C.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream)))
    return labels, mu, passes.value


def profile_enable(on: bool = True, family: str | None = None) -> None:
    """Start (clearing the counters) or stop per-kernel-family event timing in the library;
    with `family`, only that family records events."""
    if on and family is not None:
        check(lib().raftgp_profile_enable_family(family.encode()))
    else:
        check(lib().raftgp_profile_enable(1 if on else 0))


def profile_read() -> dict:
    """{family: {"launches", "timed", "ms"}} since the last profile_enable(True)."""
    buf = (_abi.ProfEntry * 32)()
    k = lib().raftgp_profile_read(buf, 32)
    return {buf[i].name.decode(): {"launches": buf[i].launches, "timed": buf[i].timed, "ms": buf[i].ms}
            for i in range(k)}


def version() -> str:
    return lib().raftgp_version().decode()


# ---- differentiation form (argument marshalling only; every step runs in the library) ----
def _diff_ws(n, width, K, device):
    return _workspace(int(lib().raftgp_diff_workspace_size(int(n), int(width), int(K))), device)


def _f32(t: torch.Tensor) -> torch.Tensor:
    if t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError("expected a contiguous float32 tensor")
    return t


def gcn_layer_forward(g: DeviceGraph, H: torch.Tensor, W: torch.Tensor, stream=None) -> torch.Tensor:
    """One Eq. 6 layer: rownorm(tanh(Ahat (H W)))."""
    H, W = _f32(H), _f32(W)
    lin, lout = W.shape
    out = torch.empty((g.n, lout), dtype=torch.float32, device=H.device)
    ws = _diff_ws(g.n, max(lin, lout), 0, H.device)
    csr = g.csr()
    check(lib().raftgp_gcn_layer_forward(C.byref(csr), C.c_void_p(H.data_ptr()), lin, C.c_void_p(W.data_ptr()), lout,
                                         C.c_void_p(out.data_ptr()), C.c_void_p(ws.data_ptr()), ws.numel(),
                                         _stream(stream)))
    return out


def gcn_layer_backward(g: DeviceGraph, H: torch.Tensor, W: torch.Tensor, dH_out: torch.Tensor, need_dH=True,
                       stream=None):
    """(dH_in or None, dW) of one layer, the forward recomputed from H."""
    H, W, dH_out = _f32(H), _f32(W), _f32(dH_out)
    lin, lout = W.shape
    dW = torch.empty((lin, lout), dtype=torch.float32, device=H.device)
    dH = torch.empty((g.n, lin), dtype=torch.float32, device=H.device) if need_dH else None
    ws = _diff_ws(g.n, max(lin, lout), 0, H.device)
    csr = g.csr()
    check(lib().raftgp_gcn_layer_backward(C.byref(csr), C.c_void_p(H.data_ptr()), lin, C.c_void_p(W.data_ptr()), lout,
                                          C.c_void_p(dH_out.data_ptr()), C.c_void_p(dH.data_ptr() if need_dH else None),
                                          C.c_void_p(dW.data_ptr()), C.c_void_p(ws.data_ptr()), ws.numel(),
                                          _stream(stream)))
    return dH, dW


def softmod_loss(g: DeviceGraph, Z: torch.Tensor, mu: torch.Tensor, tau: float, need_grad=True, stream=None):
    """(loss as a Python float, dL/dZ or None) of the relaxed soft-assignment modularity."""
    Z, mu = _f32(Z), _f32(mu)
    d = Z.shape[1]
    K = mu.shape[0]
    dZ = torch.empty_like(Z) if need_grad else None
    ws = _diff_ws(g.n, d, K, Z.device)
    loss = C.c_double(0.0)
    csr = g.csr()
    check(lib().raftgp_softmod_loss(C.byref(csr), C.c_void_p(Z.data_ptr()), d, C.c_void_p(mu.data_ptr()), K,
                                    float(tau), C.byref(loss), C.c_void_p(dZ.data_ptr() if need_grad else None),
                                    C.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream)))
    return loss.value, dZ


def centroids(Z: torch.Tensor, labels: torch.Tensor, K: int, stream=None) -> torch.Tensor:
    Z = _f32(Z)
    n, d = Z.shape
    lab = labels.to(torch.int32).contiguous()
    mu = torch.empty((K, d), dtype=torch.float32, device=Z.device)
    ws = _diff_ws(n, d, K, Z.device)
    check(lib().raftgp_centroids(C.c_void_p(Z.data_ptr()), n, d, C.c_void_p(lab.data_ptr()), int(K),
                                 C.c_void_p(mu.data_ptr()), C.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream)))
    return mu


def adam_step(param: torch.Tensor, grad: torch.Tensor, m: torch.Tensor, v: torch.Tensor, step: int, lr=1e-3,
              beta1=0.9, beta2=0.999, eps=1e-8, stream=None) -> None:
    for t in (param, grad, m, v):
        _f32(t)
    check(lib().raftgp_adam_step(C.c_void_p(param.data_ptr()), C.c_void_p(grad.data_ptr()), C.c_void_p(m.data_ptr()),
                                 C.c_void_p(v.data_ptr()), param.numel(), float(lr), float(beta1), float(beta2),
                                 float(eps), int(step), _stream(stream)))


class DiffPlan:
    """The differentiation form's calls against a graph checked once: creation validates the
    graph and computes its normalisation (one synchronisation); every later call is
    asynchronous, and the loss stays on the device.  The calls share the plan's workspace, so
    they run in order on one stream.  `width` bounds the layer widths and d, `K` the centroid
    count."""

    def __init__(self, g: DeviceGraph, width: int, K: int = 0, stream=None):
        self.g = g
        self.width, self.K = int(width), int(K)
        dev = g.col.device
        self.ws = torch.empty(int(lib().raftgp_diff_workspace_size(g.n, self.width, self.K)), dtype=torch.uint8,
                              device=dev)
        h = C.c_void_p()
        csr = g.csr()
        check(lib().raftgp_diff_plan_create(C.byref(csr), self.width, self.K, C.c_void_p(self.ws.data_ptr()),
                                            self.ws.numel(), _stream(stream), C.byref(h)))
        self._h = h

    def layer_forward(self, H: torch.Tensor, W: torch.Tensor, stream=None) -> torch.Tensor:
        H, W = _f32(H), _f32(W)
        lin, lout = W.shape
        out = torch.empty((self.g.n, lout), dtype=torch.float32, device=H.device)
        check(lib().raftgp_diff_plan_layer_forward(self._h, C.c_void_p(H.data_ptr()), lin, C.c_void_p(W.data_ptr()),
                                                   lout, C.c_void_p(out.data_ptr()), _stream(stream)))
        return out

    def layer_backward(self, H: torch.Tensor, W: torch.Tensor, dH_out: torch.Tensor, need_dH=True, stream=None):
        H, W, dH_out = _f32(H), _f32(W), _f32(dH_out)
        lin, lout = W.shape
        dW = torch.empty((lin, lout), dtype=torch.float32, device=H.device)
        dH = torch.empty((self.g.n, lin), dtype=torch.float32, device=H.device) if need_dH else None
        check(lib().raftgp_diff_plan_layer_backward(self._h, C.c_void_p(H.data_ptr()), lin, C.c_void_p(W.data_ptr()),
                                                    lout, C.c_void_p(dH_out.data_ptr()),
                                                    C.c_void_p(dH.data_ptr() if need_dH else None),
                                                    C.c_void_p(dW.data_ptr()), _stream(stream)))
        return dH, dW

    def softmod_loss(self, Z: torch.Tensor, mu: torch.Tensor, tau: float, need_grad=True, stream=None):
        """(loss as a 0-dim float64 device tensor, dL/dZ or None)."""
        Z, mu = _f32(Z), _f32(mu)
        loss = torch.empty((), dtype=torch.float64, device=Z.device)
        dZ = torch.empty_like(Z) if need_grad else None
        check(lib().raftgp_diff_plan_softmod_loss(self._h, C.c_void_p(Z.data_ptr()), Z.shape[1],
                                                  C.c_void_p(mu.data_ptr()), mu.shape[0], float(tau),
                                                  C.c_void_p(loss.data_ptr()),
                                                  C.c_void_p(dZ.data_ptr() if need_grad else None), _stream(stream)))
        return loss, dZ

    def close(self):
        if getattr(self, "_h", None):
            lib().raftgp_diff_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gcn_weights(layer: int, lin: int, lout: int, seed: int, device, stream=None) -> torch.Tensor:
    """The Eq. 6 weights the embedding draws for `layer` (1-based) from `seed`."""
    W = torch.empty((lin, lout), dtype=torch.float32, device=device)
    check(lib().raftgp_gcn_weights(int(layer), int(lin), int(lout), int(seed), C.c_void_p(W.data_ptr()),
                                   _stream(stream)))
    return W


# ---- many graphs at once ----
def concat_graphs(graphs, device, row_ptr_bits=64):
    """One block-diagonal DeviceGraph of host graphs (row_ptr, col) and the node offsets."""
    import numpy as np
    offs = [0]
    rps, cols = [], []
    e0 = 0
    for g in graphs:
        rp = np.asarray(g.row_ptr, dtype=np.int64)
        rps.append(rp[:-1] + e0)
        cols.append(np.asarray(g.col, dtype=np.int64) + offs[-1])
        e0 += int(rp[-1])
        offs.append(offs[-1] + g.n)
    rp = np.concatenate(rps + [np.array([e0], dtype=np.int64)])
    col = np.concatenate(cols).astype(np.int32)
    rdt = torch.int64 if row_ptr_bits == 64 else torch.int32
    dg = DeviceGraph(offs[-1], torch.tensor(rp, dtype=rdt, device=device), torch.tensor(col, device=device))
    return dg, np.asarray(offs, dtype=np.int64)


def batch_opts(kmin=2, kmax_factor=2.0, grid=10, iters=50, criterion="mod", seed=2, lloyd_variant=0, assign="ffma",
               embed_variant=0):
    o = _abi.BatchOpts()
    o.kmin, o.kmax_factor, o.grid, o.iters = int(kmin), float(kmax_factor), int(grid), int(iters)
    o.criterion = _abi.CRIT[criterion] if isinstance(criterion, str) else int(criterion)
    o.lloyd_variant = int(lloyd_variant)
    o.embed_variant = int(embed_variant)
    o.assign = _code(_abi.ASSIGN, assign)
    o.seed = int(seed)
    return o


class BatchPlan:
    """A captured partition of many graphs (one block-diagonal CSR): run() replays it."""

    def __init__(self, g: DeviceGraph, graph_off, dims=(64, 64, 32), dtype="f32", embed_seed=1, theta=None, W=None,
                 stream=None, op="ncut", **kw):
        import numpy as np
        self.g = g
        self.off = np.ascontiguousarray(graph_off, dtype=np.int64)
        self.ng = len(self.off) - 1
        dev = g.col.device
        if theta is not None:
            theta = theta.to(dev, torch.float32).contiguous()
        if W is not None:
            W = [w.to(dev, torch.float32).contiguous() for w in W]
        self._keep = (theta, W)
        self.eo = embed_opts(op, dims, _dtype_code(dtype), embed_seed, theta, W)
        self.bo = batch_opts(**kw)
        self.csr = g.csr()
        offp = self.off.ctypes.data_as(C.POINTER(C.c_int64))
        nbytes = lib().raftgp_batch_workspace_size(C.byref(self.csr), offp, self.ng, C.byref(self.eo), C.byref(self.bo))
        if nbytes == 0:
            raise _abi.RaftgpError(_abi.EINVAL, "invalid batch: " + lib().raftgp_last_error().decode())
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        self.labels = torch.empty(g.n, dtype=torch.int32, device=dev)
        self.k = torch.empty(self.ng, dtype=torch.int32, device=dev)
        h = C.c_void_p()
        check(lib().raftgp_batch_plan_create(C.byref(self.csr), offp, self.ng, C.byref(self.eo), C.byref(self.bo),
                                             C.c_void_p(self.labels.data_ptr()), C.c_void_p(self.k.data_ptr()),
                                             C.c_void_p(self.ws.data_ptr()), self.ws.numel(), _stream(stream),
                                             C.byref(h)))
        self._h = h

    def run(self, stream=None):
        check(lib().raftgp_batch_plan_run(self._h, _stream(stream)))
        return self.labels, self.k

    def candidates(self):
        import numpy as np
        n = self.ng * _abi.BATCH_SLOTS
        k = np.zeros(n, dtype=np.int32)
        mod = np.zeros(n)
        ncut = np.zeros(n)
        passes = np.zeros(n, dtype=np.int32)
        check(lib().raftgp_batch_plan_candidates(self._h, C.c_void_p(k.ctypes.data), C.c_void_p(mod.ctypes.data),
                                                 C.c_void_p(ncut.ctypes.data), C.c_void_p(passes.ctypes.data)))
        shp = (self.ng, _abi.BATCH_SLOTS)
        return k.reshape(shp), mod.reshape(shp), ncut.reshape(shp), passes.reshape(shp)

    def tuning(self):
        th, pp = C.c_int32(), C.c_int32()
        ms = (C.c_float * 7)()
        check(lib().raftgp_batch_plan_tuning(self._h, C.byref(th), C.byref(pp), ms))
        fv = C.c_int32()
        fms = (C.c_float * 4)()
        check(lib().raftgp_batch_plan_tuning_embed(self._h, C.byref(fv), fms))
        return {"threads": th.value, "points_per_thread": pp.value, "ms": list(ms),
                "embed_gather_variant": fv.value, "embed_gather_ms": list(fms)}

    def check(self):
        """Synchronises and raises if a bounded device wait of the last replay gave up."""
        check(lib().raftgp_batch_plan_check(self._h))

    def embedding(self):
        """The embedding of the last replay (n x d, the plan's dtype)."""
        d = self.eo.dims[self.eo.n_layers]
        Z = torch.empty((self.g.n, d), dtype=_torch_dtype(self.eo.dtype), device=self.g.col.device)
        check(lib().raftgp_batch_plan_embedding(self._h, C.c_void_p(Z.data_ptr())))
        return Z

    def close(self):
        if getattr(self, "_h", None):
            lib().raftgp_batch_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- Algorithm 1 ----
READING = {"literal": 0, "global": 1}


def _bisect_opts(eps, iters, reading, seed):
    o = _abi.BisectOpts()
    o.eps, o.iters, o.seed = int(eps), int(iters), int(seed)
    o.reading = READING[reading] if isinstance(reading, str) else int(reading)
    return o


def select_bisect(g: DeviceGraph, Z: torch.Tensor, eps=5, iters=50, reading="literal", seed=2, stream=None,
                  return_leaf=False):
    """Algorithm 1 (recursive bisection by local modularity): returns (labels int32[N], K), and
    the leaf ids (uint64 tree node of each node's block, as int64) with return_leaf."""
    n, d = Z.shape
    code = 1 if Z.dtype == torch.bfloat16 else 0
    o = _bisect_opts(eps, iters, reading, seed)
    Zc = Z.contiguous()
    labels = torch.empty(n, dtype=torch.int32, device=Z.device)
    leaf = torch.empty(n, dtype=torch.int64, device=Z.device)
    ws = _workspace(int(lib().raftgp_bisect_workspace_size(n, d, int(eps))), Z.device)
    k = C.c_int32(0)
    csr = g.csr()
    check(lib().raftgp_select_bisect(C.byref(csr), C.c_void_p(Zc.data_ptr()), d, code, C.byref(o),
                                     C.c_void_p(labels.data_ptr()), C.c_void_p(leaf.data_ptr()), C.byref(k),
                                     C.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream)))
    return (labels, k.value, leaf) if return_leaf else (labels, k.value)


def select_bisect_update(g: DeviceGraph, Z: torch.Tensor, old_labels: torch.Tensor, old_k: int, old_leaf: torch.Tensor,
                         changed: torch.Tensor, eps=5, iters=50, reading="literal", seed=2, stream=None):
    """Streaming update of Algorithm 1 (Section III-D) on the new graph and embedding, reusing
    the previous tree where no node changed: returns (labels, K, leaf ids)."""
    n, d = Z.shape
    code = 1 if Z.dtype == torch.bfloat16 else 0
    o = _bisect_opts(eps, iters, reading, seed)
    Zc = Z.contiguous()
    dev = Z.device
    old_labels = old_labels.to(dev, torch.int32).contiguous()
    old_leaf = old_leaf.to(dev, torch.int64).contiguous()
    changed = changed.to(dev, torch.uint8).contiguous()
    labels = torch.empty(n, dtype=torch.int32, device=dev)
    leaf = torch.empty(n, dtype=torch.int64, device=dev)
    ws = _workspace(int(lib().raftgp_bisect_workspace_size(n, d, int(eps))), dev)
    k = C.c_int32(0)
    csr = g.csr()
    check(lib().raftgp_select_bisect_update(C.byref(csr), C.c_void_p(Zc.data_ptr()), d, code, C.byref(o),
                                            C.c_void_p(old_labels.data_ptr()), int(old_k),
                                            C.c_void_p(old_leaf.data_ptr()), C.c_void_p(changed.data_ptr()),
                                            C.c_void_p(labels.data_ptr()), C.c_void_p(leaf.data_ptr()), C.byref(k),
                                            C.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream)))
    return labels, k.value, leaf


# ---- Algorithm 2: graphs from the SBM of Definition 1 (argument marshalling only) ----
def sbm_sample(block: torch.Tensor, theta: torch.Tensor, omega: torch.Tensor, seed=0, weights=False, stream=None):
    """One draw of an undirected graph from the degree-corrected SBM (A_ij ~ Pois(theta_i
    theta_j Omega_{c_i c_j}), i < j) by Algorithm 2 on the device: returns (src, dst) int32
    edge lists (and the values A_ij >= 1 with weights=True) in the order (block pair,
    segment, draw)."""
    dev = block.device
    blk = block.to(torch.int32).contiguous()
    th = theta.to(torch.float64).contiguous()
    om = omega.to(torch.float64).contiguous()
    p = _abi.Sbm()
    p.n, p.k, p.seed = int(blk.numel()), int(om.shape[0]), int(seed)
    p.block, p.theta, p.omega = blk.data_ptr(), th.data_ptr(), om.data_ptr()
    ws = _workspace(int(lib().raftgp_sbm_workspace_size(p.n, p.k)), dev)
    m = C.c_int64(0)
    check(lib().raftgp_sbm_count(C.byref(p), C.byref(m), C.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream)))
    src = torch.empty(max(m.value, 1), dtype=torch.int32, device=dev)
    dst = torch.empty(max(m.value, 1), dtype=torch.int32, device=dev)
    w = torch.empty(max(m.value, 1), dtype=torch.int32, device=dev) if weights else None
    check(lib().raftgp_sbm_emit(C.byref(p), C.c_void_p(src.data_ptr()), C.c_void_p(dst.data_ptr()),
                                C.c_void_p(w.data_ptr()) if weights else None, m.value, C.c_void_p(ws.data_ptr()),
                                ws.numel(), _stream(stream)))
    src, dst = src[:m.value], dst[:m.value]
    return (src, dst, w[:m.value]) if weights else (src, dst)


def coo_to_csr(n: int, src: torch.Tensor, dst: torch.Tensor, stream=None) -> DeviceGraph:
    """The symmetric CSR (int64 row_ptr, every row sorted) of undirected edges (src, dst)."""
    dev = src.device
    m = int(src.numel())
    row_ptr = torch.empty(n + 1, dtype=torch.int64, device=dev)
    col = torch.empty(max(2 * m, 1), dtype=torch.int32, device=dev)
    ws = _workspace(int(lib().raftgp_coo_to_csr_workspace_size(n)), dev)
    s32, d32 = src.to(torch.int32).contiguous(), dst.to(torch.int32).contiguous()
    check(lib().raftgp_coo_to_csr(int(n), m, C.c_void_p(s32.data_ptr()), C.c_void_p(d32.data_ptr()),
                                  C.c_void_p(row_ptr.data_ptr()), C.c_void_p(col.data_ptr()),
                                  C.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream)))
    return DeviceGraph(int(n), row_ptr, col[:2 * m])


# ---- streaming updates (Section III-D; argument marshalling only) ----
class Stream:
    """A graph and its FP32 NCut embedding kept on the device; add_edges() recomputes only the
    rows whose values change (the result equals a full embedding of the new graph)."""

    def __init__(self, g: DeviceGraph, dims=(64, 64, 32), seed=1, nnz_cap=None, W=None, stream=None, op="ncut",
                 dtype="f32"):
        self.device = g.col.device
        self.dims = tuple(dims)
        self.n = g.n
        self._h = C.c_void_p()
        if W is not None:
            W = [w.to(self.device, torch.float32).contiguous() for w in W]
        self._W = W
        self._o = embed_opts(op, dims, dtype, seed, None, W, None)
        cap = int(nnz_cap if nnz_cap is not None else 2 * g.nnz + 1024)
        nbytes = int(lib().raftgp_stream_workspace_size(g.n, cap, C.byref(self._o)))
        self._ws = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=self.device)   # owned by this stream
        csr = g.csr()
        check(lib().raftgp_stream_create(C.byref(csr), C.byref(self._o), cap, C.c_void_p(self._ws.data_ptr()),
                                         self._ws.numel(), C.byref(self._h), _stream(stream)))

    def add_edges(self, src: torch.Tensor, dst: torch.Tensor, stream=None):
        s = src.to(self.device, torch.int32).contiguous()
        d = dst.to(self.device, torch.int32).contiguous()
        check(lib().raftgp_stream_add_edges(self._h, C.c_void_p(s.data_ptr()), C.c_void_p(d.data_ptr()),
                                            int(s.numel()), _stream(stream)))
        return self.affected()

    def _info(self):
        n, nnz = C.c_int64(0), C.c_int64(0)
        aff = (C.c_int64 * (_abi.MAX_LAYERS + 1))()
        check(lib().raftgp_stream_info(self._h, C.byref(n), C.byref(nnz), aff))
        return n.value, nnz.value, [aff[k] for k in range(len(self.dims))]

    def affected(self):
        """Rows recomputed by the last update, per stage (projection, then each GCN layer)."""
        return self._info()[2]

    def graph(self, stream=None) -> DeviceGraph:
        """A copy of the current graph (int64 row pointers, sorted rows)."""
        n, nnz, _ = self._info()
        rp = torch.empty(n + 1, dtype=torch.int64, device=self.device)
        col = torch.empty(max(nnz, 1), dtype=torch.int32, device=self.device)
        check(lib().raftgp_stream_copy(self._h, C.c_void_p(rp.data_ptr()), C.c_void_p(col.data_ptr()), None,
                                       _stream(stream)))
        return DeviceGraph(n, rp, col[:nnz])

    def embedding(self, stream=None) -> torch.Tensor:
        """A copy of the current Z (n x dims[-1], FP32)."""
        Z = torch.empty((self.n, self.dims[-1]), dtype=torch.float32, device=self.device)
        check(lib().raftgp_stream_copy(self._h, None, None, C.c_void_p(Z.data_ptr()), _stream(stream)))
        return Z

    def close(self):
        if getattr(self, "_h", None):
            lib().raftgp_stream_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
