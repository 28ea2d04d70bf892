"""Seeded synthetic degree-corrected SBM graphs (input preparation only).

This module builds the inputs that both the CUDA path and the CPU oracle consume.
It holds none of RaftGP's own arithmetic (no projection, GCN, k-means or scoring):
it only draws graphs from the degree-corrected stochastic block model of Def. 4
(A_ij ~ Pois(theta_i theta_j Omega_{c_i c_j})), collapsed to a simple undirected
graph as the problem statement of Section II requires (unweighted, no self loops).

Recipe (one graph):
  1. block sizes ~ Multinomial(N, Dirichlet(alpha * 1_K)), redrawn until no block is empty;
  2. theta_i from a continuous power law x^-gamma truncated to [dmin, dmax]
     (inverse CDF);
  3. Omega_rr = a / kappa_r, Omega_rs = b (r != s), kappa_r = sum_{i in r} theta_i,
     with a, b solved so that the expected within/between edge ratio and the
     expected mean degree hit their targets;
  4. per block pair, a Poisson total with endpoints drawn proportionally to theta
     (Poisson splitting: the same law as independent Pois(lambda_ij) per pair,
     the distribution that Algorithm 2 samples exactly);
  5. multi-edges collapsed to one, self loops dropped, both directions stored;
  6. node ids randomly permuted so no locality is handed to the kernels.

Everything is vectorised numpy and driven by one PCG64 seed.
"""
from __future__ import annotations

from dataclasses import dataclass
import numpy as np


@dataclass
class Graph:
    """Symmetric CSR of a simple undirected graph plus its planted blocks."""
    n: int
    row_ptr: np.ndarray      # int64[n+1]
    col: np.ndarray          # int32[nnz], sorted within each row
    planted: np.ndarray      # int32[n], planted block of each node
    k_planted: int

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def n_edges(self) -> int:
        """Undirected edge count |E| (each edge is stored twice in the CSR)."""
        return self.nnz // 2

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr)


def _sorted_unique(a):
    a = np.sort(a)
    if a.size == 0:
        return a
    return a[np.concatenate([[True], a[1:] != a[:-1]])]


def _power_law(rng, n, gamma, lo, hi):
    u = rng.random(n)
    e = 1.0 - gamma
    return (lo ** e + u * (hi ** e - lo ** e)) ** (1.0 / e)


def _block_sizes(rng, n, k, alpha):
    for _ in range(1000):
        p = rng.dirichlet(np.full(k, float(alpha)))
        sizes = rng.multinomial(n, p)
        if (sizes > 0).all():
            return sizes
    raise ValueError("could not draw non-empty blocks; lower K or raise alpha")


def dcsbm(n: int, k: int, *, alpha: float = 5.0, gamma: float = 2.5, dmin: float = 5.0,
          dmax: float = 100.0, mean_degree: float = 16.0, ratio: float = 5.0,
          seed: int = 0) -> Graph:
    """Draw one degree-corrected SBM graph (see the module docstring for the recipe)."""
    if n < 1 or k < 1 or k > n:
        raise ValueError("need 1 <= k <= n")
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = _block_sizes(rng, n, k, alpha)
    block_of_sorted = np.repeat(np.arange(k, dtype=np.int64), sizes)   # nodes sorted by block
    theta = _power_law(rng, n, gamma, dmin, dmax)
    start = np.concatenate([[0], np.cumsum(sizes)])
    kappa = np.add.reduceat(theta, start[:-1])
    S = kappa.sum()
    total = n * mean_degree / 2.0
    within = total * ratio / (1.0 + ratio)
    between = total / (1.0 + ratio)
    a = 2.0 * within / S
    denom = S * S - np.sum(kappa * kappa)
    b = 2.0 * between / denom if denom > 0 else 0.0

    # Poisson totals per block pair (r <= s).  Within block r: ordered endpoint pairs
    # drawn with total rate a*kappa_r/2 give each unordered pair rate theta_i theta_j a/kappa_r.
    r_idx, s_idx = np.triu_indices(k)
    lam = np.where(r_idx == s_idx, a * kappa[r_idx] / 2.0, b * kappa[r_idx] * kappa[s_idx])
    counts = rng.poisson(lam)
    m = int(counts.sum())
    er = np.repeat(r_idx, counts)
    es = np.repeat(s_idx, counts)

    cum = np.concatenate([[0.0], np.cumsum(theta)])     # global cumulative theta, nodes sorted by block

    def draw(blocks):
        lo = cum[start[blocks]]
        u = rng.random(blocks.shape[0])
        x = lo + u * kappa[blocks]
        idx = np.searchsorted(cum, x, side="right") - 1
        # keep the draw inside its block even at the floating-point edges
        return np.clip(idx, start[blocks], start[blocks + 1] - 1)

    ii = draw(er)
    jj = draw(es)
    keep = ii != jj
    ii, jj = ii[keep], jj[keep]
    lo_ = np.minimum(ii, jj)
    hi_ = np.maximum(ii, jj)
    key = _sorted_unique(lo_ * np.int64(n) + hi_)
    u_ = key // n
    v_ = key % n

    perm = rng.permutation(n).astype(np.int64)          # sorted position -> public node id
    planted = np.empty(n, dtype=np.int32)
    planted[perm] = block_of_sorted.astype(np.int32)
    return _csr_from_unique_pairs(n, perm[u_], perm[v_], planted, k)


def dcsbm_params(n: int, k: int, *, alpha: float = 5.0, gamma: float = 2.5, dmin: float = 5.0,
                 dmax: float = 100.0, mean_degree: float = 16.0, ratio: float = 5.0, seed: int = 0):
    """The model of steps 1-3 of the recipe as the parameters of Definition 1 (for a sampler
    that draws the graph itself): block[i] (int32, node ids randomly permuted), theta[i]
    (float64) and Omega (K x K float64; Omega_rr = a / kappa_r, Omega_rs = b)."""
    if n < 1 or k < 1 or k > n:
        raise ValueError("need 1 <= k <= n")
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = _block_sizes(rng, n, k, alpha)
    block_of_sorted = np.repeat(np.arange(k, dtype=np.int64), sizes)
    theta = _power_law(rng, n, gamma, dmin, dmax)
    start = np.concatenate([[0], np.cumsum(sizes)])
    kappa = np.add.reduceat(theta, start[:-1])
    S = kappa.sum()
    total = n * mean_degree / 2.0
    a = 2.0 * (total * ratio / (1.0 + ratio)) / S
    denom = S * S - np.sum(kappa * kappa)
    b = 2.0 * (total / (1.0 + ratio)) / denom if denom > 0 else 0.0
    omega = np.full((k, k), b)
    np.fill_diagonal(omega, a / kappa)
    perm = rng.permutation(n).astype(np.int64)          # sorted position -> public node id
    block = np.empty(n, dtype=np.int32)
    block[perm] = block_of_sorted.astype(np.int32)
    th = np.empty(n, dtype=np.float64)
    th[perm] = theta
    return block, th, omega


def _csr_from_unique_pairs(n, u, v, planted, k_planted):
    """Symmetric CSR from distinct undirected pairs u != v (each listed once)."""
    src = np.concatenate([u, v])
    dst = np.concatenate([v, u])
    key = np.sort(src * np.int64(max(n, 1)) + dst)
    src = key // max(n, 1)
    dst = key - src * max(n, 1)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(src, minlength=n), out=row_ptr[1:])
    return Graph(n=n, row_ptr=row_ptr, col=dst.astype(np.int32), planted=np.asarray(planted, np.int32),
                 k_planted=int(k_planted))


def from_edges(n: int, u, v, *, planted=None, k_planted: int = 0) -> Graph:
    """Symmetric CSR from an undirected edge list (duplicates and self loops removed)."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    keep = u != v
    u, v = u[keep], v[keep]
    lo_ = np.minimum(u, v)
    hi_ = np.maximum(u, v)
    key = _sorted_unique(lo_ * np.int64(max(n, 1)) + hi_)
    if planted is None:
        planted = np.zeros(n, dtype=np.int32)
    return _csr_from_unique_pairs(n, key // max(n, 1), key % max(n, 1), planted, k_planted)


# The workloads the tests and the benchmark use (sizes from the method's evaluation
# settings: K grows like N^0.35, power-law degree propensities, planted block ratio).
WORKLOADS = {
    # N=1,000, K=11, Dirichlet(5) sizes, degree exponent 2.5 in [5,100], mean degree 16, 5:1.
    "dcsbm-1k": dict(n=1_000, k=11, alpha=5.0, gamma=2.5, dmin=5, dmax=100, mean_degree=16, ratio=5.0),
    # N=50,000, K=44, Dirichlet(2), exponent 2.5 in [5,500], mean degree 20, 3:1.
    "dcsbm-50k": dict(n=50_000, k=44, alpha=2.0, gamma=2.5, dmin=5, dmax=500, mean_degree=20, ratio=3.0),
    # N=1,000,000, K=200, Dirichlet(1), exponent 2.2 in [5,5000], mean degree 25, 2:1.
    "dcsbm-1m": dict(n=1_000_000, k=200, alpha=1.0, gamma=2.2, dmin=5, dmax=5000, mean_degree=25, ratio=2.0),
    # N=200,000, K=80, Dirichlet(2), exponent 2.5 in [5,500], mean degree 20, 2:1.
    "dcsbm-200k": dict(n=200_000, k=80, alpha=2.0, gamma=2.5, dmin=5, dmax=500, mean_degree=20, ratio=2.0),
    # N=2,000, K=8: the gradient-check graph of the differentiable form.
    "dcsbm-2k": dict(n=2_000, k=8, alpha=2.0, gamma=2.5, dmin=5, dmax=100, mean_degree=20, ratio=2.0),
}


def fingerprint(g: Graph) -> str:
    """SHA-256 of the CSR arrays (little-endian int64 row_ptr, then int32 col): identifies a
    generated graph, so stored results can be matched to the graph they were computed on."""
    import hashlib
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(g.row_ptr, dtype="<i8").tobytes())
    h.update(np.ascontiguousarray(g.col, dtype="<i4").tobytes())
    return h.hexdigest()


def workload(name: str, seed: int = 0) -> Graph:
    return dcsbm(seed=seed, **WORKLOADS[name])


def batch_workload(n_graphs: int = 512, seed: int = 4000, n_lo: int = 1_000, n_hi: int = 50_000):
    """Many uneven graphs: N log-uniform in [n_lo, n_hi], K = round(N^0.35), exponent 2.5,
    mean degree uniform in [10, 30], within:between ratio uniform in [2, 6]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    graphs = []
    for g in range(n_graphs):
        n = int(round(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi)))))
        k = max(2, int(round(n ** 0.35)))
        md = float(rng.uniform(10, 30))
        ratio = float(rng.uniform(2, 6))
        graphs.append(dcsbm(n, k, alpha=2.0, gamma=2.5, dmin=5, dmax=min(500.0, n / 4),
                            mean_degree=md, ratio=ratio, seed=seed * 1000 + g))
    return graphs
