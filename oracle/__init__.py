"""FP64 CPU oracle for RaftGP's hot path -- TEST INFRASTRUCTURE ONLY.

Thin ctypes marshalling around ``raftgp_oracle.c`` (a plain single-threaded FP64 C
restatement of Section III of the paper: Eq. 5 projection, Eq. 6 GCN with row
l2-normalisation, k-means model selection scored by Eq. 1 / Eq. 3 / Eq. 7).
Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may
import this package; the library path never does.  It shares no code with the CUDA
library.  Build with ``python -m oracle.build`` (``__graft_entry__.build()`` does it too).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

OP_NCUT, OP_MOD_FULL, OP_MOD_REDUCED = 0, 1, 2
CRIT_MOD, CRIT_NCUT = 0, 1
OPS = {"ncut": OP_NCUT, "mod_full": OP_MOD_FULL, "mod_reduced": OP_MOD_REDUCED}

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.library_path()
        if not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_build.SOURCE):
            _build.build()
        _lib = C.CDLL(path)
    return _lib


def _p(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _csr(g):
    return (C.c_int64(int(g.n)), _p(np.ascontiguousarray(g.row_ptr, np.int64), C.c_int64),
            _p(np.ascontiguousarray(g.col, np.int32), C.c_int32))


def _keep(g):
    # keep contiguous copies alive for the duration of a call
    return np.ascontiguousarray(g.row_ptr, np.int64), np.ascontiguousarray(g.col, np.int32)


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with status {rc}")


def set_threads(n=0):
    """Threads for the oracle's parallel loops (0: one per processor); returns the count in
    effect.  Results are bit-identical for any count."""
    return int(lib().orc_set_threads(C.c_int(int(n))))


def has_openmp():
    return bool(lib().orc_openmp())


def philox4x32_10(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c, C.c_uint32), _p(k, C.c_uint32), _p(out, C.c_uint32))
    return out


def theta(n_or_rows, L, seed):
    """Eq. 5 projection matrix rows (all rows 0..n-1 for an int, else the listed rows)."""
    if np.isscalar(n_or_rows):
        rows, nr = None, int(n_or_rows)
    else:
        rows = np.ascontiguousarray(n_or_rows, dtype=np.int64)
        nr = rows.shape[0]
    out = np.zeros((nr, L), dtype=np.float64)
    lib().orc_theta_rows(_p(rows, C.c_int64) if rows is not None else None, C.c_int64(nr), C.c_int(L),
                         C.c_uint64(seed), _p(out, C.c_double))
    return out


def gcn_weight(layer, lin, lout, seed):
    W = np.zeros((lin, lout), dtype=np.float64)
    lib().orc_gcn_weight(C.c_int(layer), C.c_int(lin), C.c_int(lout), C.c_uint64(seed), _p(W, C.c_double))
    return W


def check_csr(g):
    rp, col = _keep(g)
    return lib().orc_check_csr(C.c_int64(g.n), _p(rp, C.c_int64), _p(col, C.c_int32)) == 0


def project(g, op, th):
    rp, col = _keep(g)
    th = _f64(th)
    L = th.shape[1]
    Y = np.zeros((g.n, L), dtype=np.float64)
    _check(lib().orc_project(C.c_int64(g.n), _p(rp, C.c_int64), _p(col, C.c_int32), C.c_int(OPS.get(op, op)),
                             _p(th, C.c_double), C.c_int(L), _p(Y, C.c_double)), "project")
    return Y


def gcn_layer(g, Zin, W):
    rp, col = _keep(g)
    Zin = _f64(Zin)
    W = _f64(W)
    Z = np.zeros((g.n, W.shape[1]), dtype=np.float64)
    _check(lib().orc_gcn_layer(C.c_int64(g.n), _p(rp, C.c_int64), _p(col, C.c_int32), _p(Zin, C.c_double),
                               C.c_int(W.shape[0]), _p(W, C.c_double), C.c_int(W.shape[1]), _p(Z, C.c_double)),
           "gcn_layer")
    return Z


def embed(g, op="ncut", dims=(64, 64, 32), seed=1, theta_in=None, W_in=None):
    """Returns (Y, Z): the Eq. 5 features and the final normalised GCN output."""
    rp, col = _keep(g)
    dims_a = np.ascontiguousarray(dims, dtype=np.int32)
    nl = len(dims) - 1
    Y = np.zeros((g.n, dims[0]), dtype=np.float64)
    Z = np.zeros((g.n, dims[-1]), dtype=np.float64)
    th = _f64(theta_in) if theta_in is not None else None
    Wc = np.concatenate([_f64(w).ravel() for w in W_in]) if W_in is not None else None
    _check(lib().orc_embed(C.c_int64(g.n), _p(rp, C.c_int64), _p(col, C.c_int32), C.c_int(OPS.get(op, op)),
                           C.c_int(nl), _p(dims_a, C.c_int32), C.c_uint64(seed),
                           _p(th, C.c_double) if th is not None else None,
                           _p(Wc, C.c_double) if Wc is not None else None, _p(Y, C.c_double),
                           _p(Z, C.c_double)), "embed")
    return Y, Z


def kmeanspp(Z, K, seed, fp32_decision=False):
    Z = _f64(Z)
    seeds = np.zeros(K, dtype=np.int64)
    _check(lib().orc_kmeanspp(_p(Z, C.c_double), C.c_int64(Z.shape[0]), C.c_int(Z.shape[1]), C.c_int(K),
                              C.c_uint64(seed), C.c_int(1 if fp32_decision else 0), _p(seeds, C.c_int64)),
           "kmeanspp")
    return seeds


def lloyd(Z, mu, T, with_objective=False):
    """Returns (labels, mu_final, passes[, objective per pass])."""
    Z = _f64(Z)
    mu = _f64(mu).copy()
    n, d = Z.shape
    labels = np.zeros(n, dtype=np.int32)
    passes = C.c_int(0)
    obj = np.zeros(T, dtype=np.float64)
    _check(lib().orc_lloyd(_p(Z, C.c_double), C.c_int64(n), C.c_int(d), C.c_int(mu.shape[0]), _p(mu, C.c_double),
                           C.c_int(T), _p(labels, C.c_int32), C.byref(passes), _p(obj, C.c_double)), "lloyd")
    if with_objective:
        return labels, mu, passes.value, obj[:passes.value]
    return labels, mu, passes.value


def score(g, labels, K):
    """Returns (m, vol, mod, ncut): per-block intra edges and volumes, Eq. 3 and Eq. 1."""
    rp, col = _keep(g)
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    m = np.zeros(K, dtype=np.int64)
    vol = np.zeros(K, dtype=np.int64)
    mod = C.c_double(0)
    ncut = C.c_double(0)
    _check(lib().orc_score(C.c_int64(g.n), _p(rp, C.c_int64), _p(col, C.c_int32), _p(lab, C.c_int32), C.c_int(K),
                           _p(m, C.c_int64), _p(vol, C.c_int64), C.byref(mod), C.byref(ncut)), "score")
    return m, vol, mod.value, ncut.value


def local_modularity(g, in_u, labels, K):
    rp, col = _keep(g)
    u = np.ascontiguousarray(in_u, dtype=np.uint8)
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    out = C.c_double(0)
    _check(lib().orc_local_modularity(C.c_int64(g.n), _p(rp, C.c_int64), _p(col, C.c_int32), _p(u, C.c_uint8),
                                      _p(lab, C.c_int32), C.c_int(K), C.byref(out)), "local_modularity")
    return out.value


def coarse_grid(kmin, kmax, G):
    out = np.zeros(G, dtype=np.int32)
    cnt = lib().orc_coarse_grid(C.c_int(kmin), C.c_int(kmax), C.c_int(G), _p(out, C.c_int32))
    return out[:cnt].tolist()


def refine_grid(lo, hi, G, done):
    d = np.ascontiguousarray(done, dtype=np.int32)
    out = np.zeros(G, dtype=np.int32)
    cnt = lib().orc_refine_grid(C.c_int(lo), C.c_int(hi), C.c_int(G), _p(d, C.c_int32), C.c_int(d.shape[0]),
                                _p(out, C.c_int32))
    return out[:cnt].tolist()


def select(g, Z, kmin, kmax, grid=0, T=50, seed=2, criterion=CRIT_MOD, seed_fp32=False):
    """Model selection; returns dict(labels, k, cands=[(K, mod, ncut, passes), ...])."""
    rp, col = _keep(g)
    Z = _f64(Z)
    cap = (kmax - kmin + 1) + 2 * grid + 2
    labels = np.zeros(g.n, dtype=np.int32)
    kb = C.c_int(0)
    nc = C.c_int(0)
    ck = np.zeros(cap, dtype=np.int32)
    cm = np.zeros(cap, dtype=np.float64)
    cn = np.zeros(cap, dtype=np.float64)
    cp = np.zeros(cap, dtype=np.int32)
    _check(lib().orc_select(C.c_int64(g.n), _p(rp, C.c_int64), _p(col, C.c_int32), _p(Z, C.c_double),
                            C.c_int(Z.shape[1]), C.c_int(kmin), C.c_int(kmax), C.c_int(grid), C.c_int(T),
                            C.c_uint64(seed), C.c_int(criterion), C.c_int(1 if seed_fp32 else 0), C.c_int(cap),
                            _p(labels, C.c_int32), C.byref(kb),
                            C.byref(nc), _p(ck, C.c_int32), _p(cm, C.c_double), _p(cn, C.c_double),
                            _p(cp, C.c_int32)), "select")
    k = nc.value
    cands = [(int(ck[i]), float(cm[i]), float(cn[i]), int(cp[i])) for i in range(k)]
    return {"labels": labels, "k": kb.value, "cands": cands}


def partition(g, op="ncut", dims=(64, 64, 32), embed_seed=1, kmin=2, kmax=40, grid=0, T=50, select_seed=2,
              criterion=CRIT_MOD):
    Y, Z = embed(g, op, dims, embed_seed)
    res = select(g, Z, kmin, kmax, grid, T, select_seed, criterion)
    res["Z"] = Z
    res["Y"] = Y
    return res


def project_rows(g, op, L, seed, rows):
    """Rows of Eq. 5's Y for a large graph (Theta rows drawn on demand)."""
    rp, col = _keep(g)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    Y = np.zeros((rows.shape[0], L), dtype=np.float64)
    _check(lib().orc_project_rows(C.c_int64(g.n), _p(rp, C.c_int64), _p(col, C.c_int32), C.c_int(OPS.get(op, op)),
                                  C.c_int(L), C.c_uint64(seed), _p(rows, C.c_int64), C.c_int64(rows.shape[0]),
                                  _p(Y, C.c_double)), "project_rows")
    return Y


def gcn_rows(g, Zin32, W, rows):
    """Rows of one Eq. 6 layer (with normalisation) from a single-precision input."""
    rp, col = _keep(g)
    Zin32 = np.ascontiguousarray(Zin32, dtype=np.float32)
    W = _f64(W)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    Z = np.zeros((rows.shape[0], W.shape[1]), dtype=np.float64)
    _check(lib().orc_gcn_rows(C.c_int64(g.n), _p(rp, C.c_int64), _p(col, C.c_int32), _p(Zin32, C.c_float),
                              C.c_int(W.shape[0]), _p(W, C.c_double), C.c_int(W.shape[1]), _p(rows, C.c_int64),
                              C.c_int64(rows.shape[0]), _p(Z, C.c_double)), "gcn_rows")
    return Z


def sbm_sample(block, theta, omega, seed, seg=65536):
    """Algorithm 2 (Section IV): one draw of the support of A ~ Pois(theta_i theta_j
    Omega_{c_i c_j}) over i < j (Definition 1), each block pair's table cut into segments of
    `seg` entries (2^16 in the library).  Returns (src, dst, weight) in the order (block
    pair, segment, draw); weight is A_ij >= 1."""
    block = np.ascontiguousarray(block, dtype=np.int32)
    theta = _f64(theta)
    omega = _f64(omega)
    n, K = block.shape[0], omega.shape[0]
    m = C.c_int64(0)
    args = (C.c_int64(n), C.c_int(K), _p(block, C.c_int32), _p(theta, C.c_double), _p(omega, C.c_double),
            C.c_uint64(seed), C.c_int64(seg))
    _check(lib().orc_sbm_sample(*args, C.c_int64(0), None, None, None, C.byref(m)), "sbm_sample")
    cnt = m.value
    src = np.zeros(cnt, np.int32)
    dst = np.zeros(cnt, np.int32)
    w = np.zeros(cnt, np.int32)
    _check(lib().orc_sbm_sample(*args, C.c_int64(cnt), _p(src, C.c_int32), _p(dst, C.c_int32), _p(w, C.c_int32),
                                C.byref(m)), "sbm_sample")
    return src, dst, w
