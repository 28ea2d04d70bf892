"""Pins of the oracle's random projection and GCN (Section III-A/B) against facts the
paper and the mathematics fix: published Philox vectors, Gaussian statistics at the
Johnson-Lindenstrauss scale, dense-matrix forms of M, Q and Q-tilde, algebraic
invariants, and closed forms of the GCN on structured graphs."""
import os

import numpy as np
import pytest
from scipy import stats

import oracle
from inputs import small
from inputs.dcsbm import workload

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle.philox4x32_10(v[0:4], v[4:6])
        assert out.tolist() == v[6:10]


def test_theta_is_gaussian_with_variance_one_over_L():
    # Eq. 5, read as variance 1/L: standardised entries must be N(0,1).
    L = 64
    th = oracle.theta(4000, L, seed=7)
    z = th.ravel() * np.sqrt(L)
    n = z.size
    assert abs(z.mean()) < 5 / np.sqrt(n)
    assert abs(z.var() - 1.0) < 5 * np.sqrt(2.0 / n)
    assert stats.kstest(z[:200000], "norm").pvalue > 1e-3
    # columns uncorrelated (catches reuse of a Philox word across columns)
    c = np.corrcoef(th[:, :8].T)
    assert np.abs(c - np.eye(8)).max() < 6 / np.sqrt(4000)


def test_theta_rows_subset_matches_full_and_depends_on_seed():
    full = oracle.theta(300, 128, seed=11)
    rows = np.array([0, 17, 299, 5])
    assert np.array_equal(oracle.theta(rows, 128, seed=11), full[rows])
    assert not np.allclose(oracle.theta(300, 128, seed=12), full)


def test_gcn_weight_xavier_scale():
    W = oracle.gcn_weight(1, 128, 64, seed=3)
    assert W.shape == (128, 64)
    assert abs(W.var() * (128 + 64) / 2 - 1.0) < 0.05
    assert not np.allclose(oracle.gcn_weight(2, 128, 64, seed=3), W)


def _degrees(g):
    return np.diff(g.row_ptr).astype(np.float64)


@pytest.mark.parametrize("seed", [0, 1])
def test_projection_matches_dense_operators(seed):
    # M = D^-1/2 A D^-1/2, Q = A - d d^T/2e (rank-one identity vs the dense matrix),
    # Q-tilde = Q on the edges only.
    g = small.random_graph(48, 0.15, seed=seed, isolated=3)
    A = small.adjacency(g)
    d = A.sum(axis=1)
    rs = np.where(d > 0, 1.0 / np.sqrt(np.maximum(d, 1)), 0.0)
    th = oracle.theta(g.n, 16, seed=5)
    M = rs[:, None] * A * rs[None, :]
    Q = A - np.outer(d, d) / d.sum()
    Qt = np.where(A > 0, Q, 0.0)
    np.testing.assert_allclose(oracle.project(g, "ncut", th), M @ th, rtol=0, atol=1e-13)
    np.testing.assert_allclose(oracle.project(g, "mod_full", th), Q @ th, rtol=0, atol=1e-12)
    np.testing.assert_allclose(oracle.project(g, "mod_reduced", th), Qt @ th, rtol=0, atol=1e-12)


def test_projection_invariants():
    g = workload("dcsbm-1k")
    d = _degrees(g)
    th = oracle.theta(g.n, 64, seed=1)
    Yq = oracle.project(g, "mod_full", th)
    # 1^T Q = 0, so every column of Q Theta sums to zero
    assert np.abs(Yq.sum(axis=0)).max() < 1e-10 * np.abs(Yq).sum(axis=0).max()
    # d^1/2 is a left eigenvector of M with eigenvalue 1
    Ym = oracle.project(g, "ncut", th)
    np.testing.assert_allclose(np.sqrt(d) @ Ym, np.sqrt(d) @ th, rtol=1e-11, atol=1e-11)


def test_projection_preserves_norms_on_average():
    # JL scale: E ||X_i Theta||^2 = ||X_i||^2 when Var(Theta_ir) = 1/L.
    g = workload("dcsbm-1k")
    d = _degrees(g)
    L = 64
    th = oracle.theta(g.n, L, seed=9)
    Y = oracle.project(g, "ncut", th)
    rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    xnorm2 = np.bincount(rows, weights=1.0 / (d[rows] * d[g.col]), minlength=g.n)
    ok = xnorm2 > 0
    ratio = (Y[ok] ** 2).sum(axis=1) / xnorm2[ok]
    assert abs(ratio.mean() - 1.0) < 6 * np.sqrt(2.0 / L / ok.sum()) * 3


def test_gcn_complete_graph_closed_form():
    # On K_n, D-hat^-1/2 (A+I) D-hat^-1/2 = J/n: every row becomes the column mean.
    g = small.complete(9)
    rng = np.random.default_rng(0)
    Zin = rng.normal(size=(9, 6))
    W = rng.normal(size=(6, 4))
    h = np.tanh(Zin.mean(axis=0) @ W)
    want = np.tile(h / np.linalg.norm(h), (9, 1))
    np.testing.assert_allclose(oracle.gcn_layer(g, Zin, W), want, atol=1e-14)


def test_gcn_edgeless_graph_closed_form():
    g = small.edgeless(5)
    rng = np.random.default_rng(1)
    Zin = rng.normal(size=(5, 3))
    W = rng.normal(size=(3, 7))
    h = np.tanh(Zin @ W)
    np.testing.assert_allclose(oracle.gcn_layer(g, Zin, W), h / np.linalg.norm(h, axis=1, keepdims=True),
                               atol=1e-14)


def test_gcn_star_closed_form():
    # Star with centre 0 and m leaves: d-hat_0 = m+1, d-hat_leaf = 2.
    m = 5
    g = small.star(m)
    rng = np.random.default_rng(2)
    Zin = rng.normal(size=(m + 1, 3))
    W = rng.normal(size=(3, 2))
    c = 1.0 / np.sqrt(2.0 * (m + 1))
    agg = np.empty_like(Zin)
    agg[0] = Zin[0] / (m + 1) + c * Zin[1:].sum(axis=0)
    agg[1:] = Zin[1:] / 2.0 + c * Zin[0]
    h = np.tanh(agg @ W)
    np.testing.assert_allclose(oracle.gcn_layer(g, Zin, W), h / np.linalg.norm(h, axis=1, keepdims=True),
                               atol=1e-14)


def test_gcn_rows_unit_norm_and_zero_row_stays_zero():
    g = small.random_graph(40, 0.1, seed=3)
    rng = np.random.default_rng(3)
    Zin = rng.normal(size=(40, 8))
    Zin[5] = 0.0
    Zin[list(g.col[g.row_ptr[5]:g.row_ptr[6]])] = 0.0   # node 5 and its neighbours all zero
    Z = oracle.gcn_layer(g, Zin, rng.normal(size=(8, 8)))
    norms = np.linalg.norm(Z, axis=1)
    assert norms[5] == 0.0
    np.testing.assert_allclose(norms[np.arange(40) != 5], 1.0, atol=1e-14)


def test_gcn_permutation_equivariance():
    g = small.random_graph(30, 0.2, seed=4)
    rng = np.random.default_rng(4)
    Zin = rng.normal(size=(30, 5))
    W = rng.normal(size=(5, 3))
    perm = rng.permutation(30)
    inv = np.argsort(perm)
    rows = np.repeat(np.arange(30), np.diff(g.row_ptr))
    from inputs.dcsbm import from_edges
    gp = from_edges(30, inv[rows], inv[g.col])
    np.testing.assert_allclose(oracle.gcn_layer(gp, Zin[perm], W), oracle.gcn_layer(g, Zin, W)[perm], atol=1e-14)


def test_embed_chains_projection_and_layers():
    g = small.random_graph(60, 0.1, seed=5)
    dims = (16, 12, 8)
    Y, Z = oracle.embed(g, "mod_full", dims, seed=3)
    th = oracle.theta(g.n, 16, seed=3)
    np.testing.assert_array_equal(Y, oracle.project(g, "mod_full", th))
    Z1 = oracle.gcn_layer(g, Y, oracle.gcn_weight(1, 16, 12, seed=3))
    Z2 = oracle.gcn_layer(g, Z1, oracle.gcn_weight(2, 12, 8, seed=3))
    np.testing.assert_array_equal(Z, Z2)


def test_row_sampled_forms_agree_with_whole_graph_forms():
    g = small.random_graph(80, 0.08, seed=6, isolated=2)
    rows = np.array([0, 5, 79, 78, 33])
    for op in ("ncut", "mod_full", "mod_reduced"):
        full = oracle.project(g, op, oracle.theta(g.n, 16, seed=4))
        np.testing.assert_allclose(oracle.project_rows(g, op, 16, 4, rows), full[rows], atol=1e-13)
    rng = np.random.default_rng(6)
    Zin = rng.normal(size=(80, 8)).astype(np.float32)
    W = rng.normal(size=(8, 4))
    np.testing.assert_allclose(oracle.gcn_rows(g, Zin, W, rows), oracle.gcn_layer(g, Zin.astype(np.float64), W)[rows],
                               atol=1e-14)


@pytest.mark.parametrize("op", ["ncut", "mod_full", "mod_reduced"])
def test_embed_without_gcn_layers_is_the_row_normalised_projection(op):
    # the "w/o Emb" ablation (Table IV): Z = rownorm(Y), a zero row stays zero
    from inputs.dcsbm import workload
    g = workload("dcsbm-1k")
    Y, Z = oracle.embed(g, op, (64,), seed=3)
    Y2, _ = oracle.embed(g, op, (64, 32), seed=3)
    assert np.array_equal(Y, Y2)                     # the same projection as with layers
    nrm = np.linalg.norm(Y, axis=1, keepdims=True)
    want = np.where(nrm > 0, Y / np.where(nrm > 0, nrm, 1.0), 0.0)
    assert np.abs(Z - want).max() <= 4e-16
    live = nrm[:, 0] > 0
    assert np.abs(np.linalg.norm(Z[live], axis=1) - 1).max() <= 1e-15
