"""Pins of the Algorithm 1 oracle (oracle/hier.py): its exact LMod against the C oracle's
Definition 5 evaluation, its K=2 seeding against the C oracle's k-means++ (tree id 0 gives
the same Philox counters), clique recovery on a ring of cliques, planted recovery on a strongly
planted DC-SBM, and the size rule on a tiny graph."""
import numpy as np

import oracle
from inputs.dcsbm import dcsbm
from inputs.small import complete, random_graph, ring_of_cliques
from oracle import hier
from paper_2312_01560_gb300.metrics import nmi


def test_exact_lmod_matches_c_oracle():
    g = random_graph(120, 0.08, 5, isolated=3)
    rng = np.random.default_rng(5)
    for K in (1, 2, 5):
        members = np.sort(rng.choice(g.n, 70, replace=False))
        lab = np.full(g.n, -1, dtype=np.int64)
        lab[members] = rng.integers(0, K, size=members.shape[0])
        num, two_e = hier.lmod_numerator(*hier.lmod_parts(g, members, lab, K))
        inu = np.zeros(g.n, dtype=np.uint8)
        inu[members] = 1
        ref = oracle.local_modularity(g, inu, np.where(lab < 0, 0, lab), K)
        assert abs(num / (two_e * two_e) - ref) <= 1e-12


def test_seeding_matches_c_kmeanspp_for_tree_id_zero():
    rng = np.random.default_rng(6)
    Z = rng.normal(size=(500, 16)).astype(np.float32)
    for seed in (1, 2, 9):
        s = hier.seeds2(Z, seed, 0)
        ref = oracle.kmeanspp(Z.astype(np.float64), 2, seed, fp32_decision=True)
        assert list(s) == list(ref)


def test_ring_of_cliques_is_recovered():
    g = ring_of_cliques(8, 12)
    rng = np.random.default_rng(7)
    truth = np.arange(g.n) // 12
    Z = (np.eye(8, 16)[truth] + 0.02 * rng.normal(size=(g.n, 16))).astype(np.float32)
    lab, K = hier.bisect(g, Z, seed=2)
    assert K == 8
    assert nmi(lab, truth) == 1.0


def test_planted_dcsbm_readings():
    # the global reading of e recovers the planted blocks; the literal one splits true blocks
    # further (halving a block with within:between ratio 12 raises its literal LMod)
    g = dcsbm(1500, 6, alpha=5.0, gamma=2.5, dmin=8, dmax=60, mean_degree=24, ratio=12.0, seed=30)
    _, Z = oracle.embed(g, "ncut", (64, 64, 32), seed=1)
    lab_g, K_g = hier.bisect(g, Z.astype(np.float32), seed=2, reading="global")
    lab_l, K_l = hier.bisect(g, Z.astype(np.float32), seed=2, reading="literal")
    print(f"global: K {K_g} NMI {nmi(lab_g, g.planted):.3f}; literal: K {K_l} NMI {nmi(lab_l, g.planted):.3f}")
    assert nmi(lab_g, g.planted) >= 0.95 and K_g == g.k_planted
    assert K_l > K_g


def test_readings_agree_at_the_root():
    g = random_graph(80, 0.1, 9)
    rng = np.random.default_rng(9)
    lab = rng.integers(0, 2, size=g.n)
    m, vb = hier.lmod_parts(g, np.arange(g.n), lab, 2)
    assert hier.lmod_numerator(m, vb) == hier.lmod_numerator(m, vb, int(g.row_ptr[-1]))


def test_small_sets_become_one_block():
    g = complete(10)
    Z = np.random.default_rng(8).normal(size=(10, 8)).astype(np.float32)
    lab, K = hier.bisect(g, Z)
    assert K == 1 and not lab.any()
