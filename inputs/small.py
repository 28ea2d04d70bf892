"""Small structured graphs with known answers (input preparation only)."""
from __future__ import annotations

import numpy as np

from .dcsbm import Graph, from_edges


def complete(n: int) -> Graph:
    u, v = np.triu_indices(n, 1)
    return from_edges(n, u, v)


def star(leaves: int) -> Graph:
    """Node 0 joined to nodes 1..leaves."""
    return from_edges(leaves + 1, np.zeros(leaves, np.int64), np.arange(1, leaves + 1))


def edgeless(n: int) -> Graph:
    return from_edges(n, np.zeros(0, np.int64), np.zeros(0, np.int64))


def ring_of_cliques(c: int, s: int) -> Graph:
    """c cliques of s nodes; clique r's last node is joined to clique r+1's first node (mod c)."""
    us, vs = [], []
    for r in range(c):
        base = r * s
        u, v = np.triu_indices(s, 1)
        us.append(u + base)
        vs.append(v + base)
        us.append(np.array([base + s - 1]))
        vs.append(np.array([((r + 1) % c) * s]))
    planted = np.repeat(np.arange(c, dtype=np.int32), s)
    return from_edges(c * s, np.concatenate(us), np.concatenate(vs), planted=planted, k_planted=c)


def random_graph(n: int, p: float, seed: int, isolated: int = 0) -> Graph:
    """Erdos-Renyi G(n, p); the last `isolated` nodes get no edges."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u, v = np.triu_indices(n, 1)
    keep = rng.random(u.shape[0]) < p
    u, v = u[keep], v[keep]
    if isolated:
        ok = (u < n - isolated) & (v < n - isolated)
        u, v = u[ok], v[ok]
    return from_edges(n, u, v)


def adjacency(g: Graph) -> np.ndarray:
    """Dense 0/1 adjacency matrix of a small graph."""
    A = np.zeros((g.n, g.n))
    rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    A[rows, g.col] = 1.0
    return A
