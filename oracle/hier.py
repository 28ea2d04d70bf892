"""FP64 oracle for Algorithm 1 (hierarchical model selection) -- TEST INFRASTRUCTURE ONLY.

Partition(U): m1 = LMod(U; G) with U as one block; K=2 k-means on {z_i : i in U} gives U1, U2;
m2 = LMod(U1, U2; G); U becomes a block if |U1| <= eps or |U2| <= eps or m1 > m2 (the stopping
test printed in Algorithm 1 names |U1| twice; the text names |U1| and |U2|), otherwise U1 and
U2 are partitioned in turn.  LMod (Definition 5, Eq. 7) with m_r the intra-block edges of U_r,
vbar_r the G-degree sum of U_r and 2e = the G-degree sum of U:
    LMod = sum_r m_r / e - (vbar_r / 2e)^2 = (2 * 2e * sum_r m_r - sum_r vbar_r^2) / (2e)^2,
compared exactly (integers).  Eq. 7 divides m_r by e while Definition 5 defines 2e as the
G-degree sum of U; both readings are here: "literal" (2e = the G-degree sum of U) and
"global" (2e = the G-degree sum of all of V, so a split is taken exactly when it raises the
graph's modularity); they agree at U = V.  K=2 k-means: k-means++ on U in ascending node order (first seed
floor(r_0 |U| / 2^64), second by D^2 sampling on floor(D^2 2^40), the D^2 decision in FP32,
direct form, ascending coordinates), then Lloyd in FP64 (the C oracle's, at most T passes).
The draws r_t are Philox4x32-10(seed; t, id_lo, id_hi, "Kmpp") words 0-1 with id the set's
node in the binary recursion tree (root 1, children 2 id and 2 id + 1); a set at depth 62 is a
block.  Blocks are labelled by increasing smallest node index.

Only the tests may import this module; the library never does."""
from __future__ import annotations

import numpy as np

from . import lloyd, philox4x32_10

STREAM_KMPP = 0x4B6D7070
MAX_DEPTH = 62


def _draw(seed, t, node_id):
    out = philox4x32_10([t, node_id & 0xFFFFFFFF, node_id >> 32, STREAM_KMPP], [seed & 0xFFFFFFFF, seed >> 32])
    return int(out[0]) | (int(out[1]) << 32)


def seeds2(Zu32, seed, node_id):
    """The two k-means++ seeds (positions in U) of a set."""
    n = Zu32.shape[0]
    s0 = (_draw(seed, 0, node_id) * n) >> 64
    c = Zu32[s0]
    d2 = np.zeros(n, dtype=np.float32)
    for k in range(Zu32.shape[1]):
        t = np.float32(Zu32[:, k] - c[k])
        d2 = np.float32(d2 + np.float32(t * t))
    q = np.floor(d2.astype(np.float64) * 2.0 ** 40).astype(np.uint64)
    cs = np.cumsum(q, dtype=np.uint64)
    tot = int(cs[-1])
    if tot == 0:
        s1 = 1 if s0 == 0 else 0
    else:
        thr = (_draw(seed, 1, node_id) * tot) >> 64
        s1 = int(np.argmax(cs > np.uint64(thr)))
    return s0, s1


def lmod_parts(g, members, labels_of, K):
    """(m_r, vbar_r) for the blocks of a set: members = node indices of U (ascending),
    labels_of = full-length array with each member's block (others ignored)."""
    rp = np.asarray(g.row_ptr, dtype=np.int64)
    col = np.asarray(g.col, dtype=np.int64)
    inu = np.zeros(g.n, dtype=bool)
    inu[members] = True
    m = [0] * K
    vb = [0] * K
    for i in members:
        r = int(labels_of[i])
        vb[r] += int(rp[i + 1] - rp[i])
        nb = col[rp[i]:rp[i + 1]]
        nb = nb[(nb > i) & inu[nb]]
        m[r] += int(np.count_nonzero(labels_of[nb] == r))
    return m, vb


def lmod_numerator(m, vb, two_e=None):
    """Numerator of LMod over (2e)^2; 2e = sum(vb) (the literal reading) unless given."""
    two_e = sum(vb) if two_e is None else two_e
    return 2 * two_e * sum(m) - sum(v * v for v in vb), two_e


def bisect(g, Z32, seed=2, eps=5, T=50, reading="literal"):
    """Algorithm 1 on embeddings Z32 (float32, N x d): returns (labels, K)."""
    Z32 = np.asarray(Z32, dtype=np.float32)
    two_e_g = int(np.asarray(g.row_ptr, dtype=np.int64)[-1]) if reading == "global" else None
    lab = np.zeros(g.n, dtype=np.int64)
    blocks = []
    stack = [(np.arange(g.n), 1, 0)]
    while stack:
        U, node_id, depth = stack.pop()
        if U.shape[0] < 2 or depth >= MAX_DEPTH:
            blocks.append(U)
            continue
        Zu = Z32[U]
        s0, s1 = seeds2(Zu, seed, node_id)
        labels, _, _ = lloyd(Zu.astype(np.float64), Zu[[s0, s1]].astype(np.float64), T)
        U1, U2 = U[labels == 0], U[labels == 1]
        lab[U] = 0
        num1, two_e = lmod_numerator(*lmod_parts(g, U, lab, 1), two_e_g)
        lab[U] = labels
        num2, _ = lmod_numerator(*lmod_parts(g, U, lab, 2), two_e_g)
        if U1.shape[0] <= eps or U2.shape[0] <= eps or (two_e > 0 and num1 > num2):
            blocks.append(U)
        else:
            # depth first: U1, then U2
            stack.append((U2, 2 * node_id + 1, depth + 1))
            stack.append((U1, 2 * node_id, depth + 1))
    blocks.sort(key=lambda b: int(b.min()))
    out = np.empty(g.n, dtype=np.int32)
    for r, b in enumerate(blocks):
        out[b] = r
    return out, len(blocks)
