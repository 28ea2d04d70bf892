"""Pins of the oracle's scoring and model selection (Section III-C; Eq. 1-4, Eq. 7)
against closed forms, brute force over every partition of a tiny graph, the matrix forms
of the objectives, a library k-means, and planted-partition recovery."""
import itertools

import numpy as np
import pytest

import oracle
from inputs import small
from inputs.dcsbm import dcsbm
from paper_2312_01560_gb300.metrics import nmi


def test_score_single_block_and_singletons():
    g = small.random_graph(30, 0.2, seed=1)
    d = np.diff(g.row_ptr).astype(np.int64)
    m, vol, mod, ncut = oracle.score(g, np.zeros(30, np.int32), 1)
    assert m[0] == g.n_edges and vol[0] == d.sum() and mod == 0.0 and ncut == 0.0
    m, vol, mod, ncut = oracle.score(g, np.arange(30, dtype=np.int32), 30)
    assert (m == 0).all() and (vol == d).all()
    assert mod == -float((d * d).sum()) / float(d.sum()) ** 2
    assert ncut == 0.5 * np.count_nonzero(d)


@pytest.mark.parametrize("c,s", [(3, 4), (5, 6), (8, 3)])
def test_score_ring_of_cliques_closed_form(c, s):
    g = small.ring_of_cliques(c, s)
    m, vol, mod, ncut = oracle.score(g, g.planted, c)
    mm = s * (s - 1) // 2
    assert (m == mm).all() and (vol == 2 * (mm + 1)).all()
    assert mod == pytest.approx(mm / (mm + 1) - 1.0 / c, abs=1e-15)
    assert ncut == pytest.approx(c / (2.0 * (mm + 1)), abs=1e-15)


def _set_partitions(n):
    # restricted growth strings: every partition of {0..n-1} once
    a = [0] * n

    def rec(i, mx):
        if i == n:
            yield list(a)
            return
        for v in range(mx + 2):
            a[i] = v
            yield from rec(i + 1, max(mx, v))

    yield from rec(1, 0)


def test_score_brute_force_against_eq3_and_matrix_forms():
    # every partition of an 8-node graph: Eq. 3 double sum, Eq. 4 trace form (modularity)
    # and Eq. 2 trace form (NCut = tr(H^T L H)/2) agree with the oracle.
    g = small.ring_of_cliques(2, 4)
    A = small.adjacency(g)
    d = A.sum(axis=1)
    two_e = d.sum()
    Q = A - np.outer(d, d) / two_e
    Lap = np.eye(8) - A / np.sqrt(np.outer(d, d))
    best = (-1.0, None)
    count = 0
    for lab in _set_partitions(8):
        lab = np.array(lab, np.int32)
        K = lab.max() + 1
        _, _, mod, ncut = oracle.score(g, lab, K)
        same = lab[:, None] == lab[None, :]
        assert mod == pytest.approx((Q * same).sum() / two_e, abs=1e-13)
        H = np.zeros((8, K))
        H[np.arange(8), lab] = 1.0
        assert mod == pytest.approx(np.trace(H.T @ Q @ H) / two_e, abs=1e-13)
        vol = H.T @ d
        Hn = H * np.sqrt(d)[:, None] / np.sqrt(vol)[None, :]
        assert ncut == pytest.approx(0.5 * np.trace(Hn.T @ Lap @ Hn), abs=1e-13)
        if mod > best[0]:
            best = (mod, lab)
        count += 1
    assert count == 4140                      # Bell(8)
    assert nmi(best[1], g.planted) == 1.0     # the optimum is the two cliques


def test_local_modularity_equals_modularity_on_whole_graph():
    g = small.random_graph(40, 0.15, seed=2)
    lab = (np.arange(40) % 3).astype(np.int32)
    _, _, mod, _ = oracle.score(g, lab, 3)
    assert oracle.local_modularity(g, np.ones(40), lab, 3) == pytest.approx(mod, abs=1e-14)


def test_local_modularity_subset_closed_form():
    # U = one clique of a ring of cliques as a single block: m = s(s-1)/2, mbar = 2m+2 = 2e_U.
    g = small.ring_of_cliques(4, 5)
    in_u = (g.planted == 0)
    mm = 10
    lm = oracle.local_modularity(g, in_u, np.zeros(g.n, np.int32), 1)
    assert lm == pytest.approx(mm / (mm + 1) - 1.0, abs=1e-15)


def test_kmeanspp_first_seed_uniform_and_second_proportional_to_d2():
    pts = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 2.0], [3.0, 1.0], [0.5, 0.5], [2.0, 2.0]])
    D2 = ((pts[:, None, :] - pts[None, :, :]) ** 2).sum(-1)
    S = 6000
    pairs = np.zeros((6, 6))
    for s in range(S):
        f, sec = oracle.kmeanspp(pts, 2, seed=s)
        pairs[f, sec] += 1
    first = pairs.sum(axis=1)
    from scipy import stats
    assert stats.chisquare(first).pvalue > 1e-3
    exp = first[:, None] * D2 / D2.sum(axis=1, keepdims=True)
    mask = exp > 0
    assert (pairs[~mask] == 0).all()          # never re-picks a chosen point
    chi = ((pairs[mask] - exp[mask]) ** 2 / exp[mask]).sum()
    assert stats.chi2.sf(chi, mask.sum() - 6) > 1e-3


def test_kmeanspp_duplicates_take_lowest_unchosen_index():
    pts = np.ones((5, 3))
    seeds = oracle.kmeanspp(pts, 4, seed=3)
    rest = [i for i in range(5) if i != seeds[0]]
    assert seeds[1:].tolist() == rest[:3]


def test_kmeanspp_fp32_decision_agrees_on_generic_data():
    rng = np.random.default_rng(5)
    Z = rng.normal(size=(500, 16))
    Z /= np.linalg.norm(Z, axis=1, keepdims=True)
    Z = Z.astype(np.float32).astype(np.float64)
    assert np.array_equal(oracle.kmeanspp(Z, 30, 9), oracle.kmeanspp(Z, 30, 9, fp32_decision=True))


def test_lloyd_matches_scipy_kmeans2():
    from scipy.cluster.vq import kmeans2
    rng = np.random.default_rng(6)
    Z = rng.normal(size=(400, 5))
    init = Z[[3, 50, 77, 200, 301, 399]]
    lab, mu, passes = oracle.lloyd(Z, init, T=100)
    # scipy does `iter` updates and then one final assignment
    cb, lab2 = kmeans2(Z, init.copy(), iter=passes, minit="matrix", missing="warn")
    assert np.array_equal(lab, lab2)
    np.testing.assert_allclose(mu, cb, atol=1e-12)


def test_lloyd_objective_non_increasing_and_k_equals_n():
    rng = np.random.default_rng(7)
    Z = rng.normal(size=(300, 4))
    _, _, passes, obj = oracle.lloyd(Z, Z[:12], T=50, with_objective=True)
    assert (np.diff(obj) <= 1e-12).all()
    lab, _, _ = oracle.lloyd(Z[:20], Z[:20], T=5)
    assert lab.tolist() == list(range(20))


def test_lloyd_empty_cluster_keeps_centroid():
    Z = np.array([[0.0], [0.1], [10.0], [10.1]])
    init = np.array([[0.0], [10.0], [100.0]])
    lab, mu, _ = oracle.lloyd(Z, init, T=10)
    assert lab.tolist() == [0, 0, 1, 1]
    assert mu[2, 0] == 100.0


def test_candidate_grids():
    assert oracle.coarse_grid(2, 100, 10) == [2, 13, 24, 35, 46, 56, 67, 78, 89, 100]
    assert oracle.coarse_grid(50, 400, 10) == [50, 89, 128, 167, 206, 244, 283, 322, 361, 400]
    assert oracle.coarse_grid(2, 5, 10) == [2, 3, 4, 5]
    assert oracle.refine_grid(13, 35, 10, [2, 13, 24, 35]) == [15, 17, 19, 21, 23, 25, 27, 29, 31, 33]
    assert oracle.refine_grid(2, 4, 10, [2, 3, 4]) == []


def test_select_ring_of_cliques_finds_cliques():
    g = small.ring_of_cliques(6, 8)
    rng = np.random.default_rng(8)
    Z = np.eye(6)[g.planted] + 0.01 * rng.normal(size=(g.n, 6))
    r = oracle.select(g, Z, 2, 12, grid=0, T=30, seed=4)
    assert r["k"] == 6 and nmi(r["labels"], g.planted) == 1.0
    assert [c[0] for c in r["cands"]] == list(range(2, 13))


def test_partition_recovers_strongly_planted_dcsbm():
    g = dcsbm(1000, 5, alpha=5.0, gamma=2.5, dmin=15, dmax=100, mean_degree=30, ratio=20.0, seed=3)
    r = oracle.partition(g, "ncut", (64, 64, 32), kmin=2, kmax=12, grid=0, T=50)
    assert r["k"] == 5
    assert nmi(r["labels"], g.planted) == 1.0


def test_hierarchical_select_refines_around_best():
    g = dcsbm(1500, 20, alpha=5.0, gamma=2.5, dmin=10, dmax=100, mean_degree=25, ratio=8.0, seed=4)
    _, Z = oracle.embed(g, "mod_full", (64, 64, 32), seed=1)
    r = oracle.select(g, Z, 2, 60, grid=10, T=50, seed=2)
    ks = [c[0] for c in r["cands"]]
    coarse = oracle.coarse_grid(2, 60, 10)
    assert ks[:len(coarse)] == coarse
    j = int(np.argmax([c[1] for c in r["cands"][:len(coarse)]]))
    lo, hi = coarse[max(j - 1, 0)], coarse[min(j + 1, len(coarse) - 1)]
    assert ks[len(coarse):] == oracle.refine_grid(lo, hi, 10, coarse)
    best = max(r["cands"], key=lambda c: (c[1], -c[0]))
    assert r["k"] == best[0]
    assert nmi(r["labels"], g.planted) > 0.95


def test_oracle_results_do_not_depend_on_thread_count():
    # the parallel loops write only their own rows, points or clusters and every floating-point
    # sum keeps its sequential order, so one thread and four give the same bits
    from inputs.dcsbm import workload
    g = workload("dcsbm-1k")
    runs = []
    for t in (1, 4):
        oracle.set_threads(t)
        Y, Z = oracle.embed(g, "mod_full", (64, 64, 32), seed=1)
        r = oracle.select(g, Z, 2, 30, grid=0, T=50, seed=2)
        _, _, _, obj = oracle.lloyd(Z, Z[:7], 20, with_objective=True)
        rows = np.arange(0, g.n, 7)
        yr = oracle.project_rows(g, "mod_full", 64, 1, rows)
        zr = oracle.gcn_rows(g, Y.astype(np.float32), oracle.gcn_weight(1, 64, 64, 1), rows)
        runs.append((Y, Z, r, obj, yr, zr))
    oracle.set_threads(0)
    (Y1, Z1, r1, o1, y1, z1), (Y4, Z4, r4, o4, y4, z4) = runs
    assert np.array_equal(Y1, Y4) and np.array_equal(Z1, Z4) and np.array_equal(o1, o4)
    assert np.array_equal(y1, y4) and np.array_equal(z1, z4)
    assert np.array_equal(y1, Y1[rows])       # the sampled rows are the whole projection's rows
    assert r1["k"] == r4["k"] and r1["cands"] == r4["cands"] and np.array_equal(r1["labels"], r4["labels"])


@pytest.mark.parametrize("name", ["dcsbm-50k", "dcsbm-1m"])
def test_stored_oracle_partition_is_consistent(name):
    # the stored partition belongs to the graph the generator draws here, its candidate scores
    # are the oracle scorer's, and K* is the best of them (exact ties to the smaller K)
    import os
    from inputs.dcsbm import fingerprint, workload
    from tests.golden.make_oracle_partitions import load, path_for
    if not os.path.exists(path_for(name)):
        pytest.skip(f"no stored oracle partition for {name}")
    ref = load(name)
    g = workload(name)
    assert fingerprint(g) == ref["fingerprint"]
    for tag in [t for t in ("", "_z32", "_zbf16") if "labels" + t in ref]:
        lab, cands, k = ref["labels" + tag], ref["cands" + tag], ref["k" + tag]
        best = max(range(len(cands)), key=lambda i: (cands[i, 1], -cands[i, 0]))
        assert int(cands[best, 0]) == k
        assert lab.min() >= 0 and lab.max() < k
        _, _, mod, ncut = oracle.score(g, lab, k)
        assert mod == cands[best, 1] and ncut == cands[best, 2]
