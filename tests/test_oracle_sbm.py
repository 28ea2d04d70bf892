"""Pins of the Algorithm 2 oracle (oracle.sbm_sample) to the law of Definition 1: every entry
i < j is nonzero with probability 1 - exp(-lambda_ij), independently, and its value given
nonzero is Pois(lambda_ij) conditioned on >= 1.  Checked by frequencies over many seeds
(z-scores), the conditional mean of the value, closed forms (no edge at Omega = 0, the
complete graph when every lambda is large), the expected edge count and its spread over the
table on graphs whose tables span several 2^16-entry segments, and the structure of the
output (no self loop, no repeated pair, endpoints ordered by block)."""
import numpy as np
import pytest

import oracle


def _lam(block, theta, om):
    return np.outer(theta, theta) * om[block][:, block]


BLOCK7 = np.array([0, 1, 0, 2, 1, 0, 1])
THETA7 = np.array([0.5, 1.0, 1.5, 2.0, 0.7, 1.2, 0.3])
OM3 = np.array([[0.8, 0.1, 0.3], [0.1, 0.5, 0.05], [0.3, 0.05, 0.6]])


@pytest.mark.parametrize("seg", [1, 2, 3, 65536])
def test_entry_frequencies_and_values_follow_the_poisson_law(seg):
    # seg = 1: every entry its own segment; 2, 3: boundaries inside every table
    n, S = 7, 6000
    lam = _lam(BLOCK7, THETA7, OM3)
    cnt = np.zeros((n, n))
    wsum = np.zeros((n, n))
    for seed in range(S):
        s, d, w = oracle.sbm_sample(BLOCK7, THETA7, OM3, seed, seg=seg)
        a, b = np.minimum(s, d), np.maximum(s, d)
        np.add.at(cnt, (a, b), 1)
        np.add.at(wsum, (a, b), w)
    iu = np.triu_indices(n, 1)
    p = 1 - np.exp(-lam[iu])
    z = (cnt[iu] / S - p) / np.sqrt(p * (1 - p) / S)
    assert np.abs(z).max() < 4.5, z
    # E[A | A >= 1] = lambda / (1 - e^-lambda), Var = (lambda + lambda^2) / (1 - e^-lambda) - mean^2
    l = lam[iu]
    c = cnt[iu]
    keep = c >= 300
    mean = l / (1 - np.exp(-l))
    var = (l + l * l) / (1 - np.exp(-l)) - mean ** 2
    zw = (wsum[iu][keep] / c[keep] - mean[keep]) / np.sqrt(var[keep] / c[keep])
    assert keep.sum() >= 10 and np.abs(zw).max() < 4.5, zw


def test_structure_of_the_output():
    rng = np.random.default_rng(3)
    n, K = 400, 6
    block = rng.integers(0, K, n)
    theta = rng.uniform(0.2, 3.0, n)
    om = rng.uniform(0.0, 0.05, (K, K))
    om = (om + om.T) / 2
    s, d, w = oracle.sbm_sample(block, theta, om, 11)
    assert len(s) > 100
    assert (s != d).all()
    assert (block[s] <= block[d]).all()
    same = block[s] == block[d]
    assert (s[same] < d[same]).all()
    pairs = set(zip(np.minimum(s, d).tolist(), np.maximum(s, d).tolist()))
    assert len(pairs) == len(s)
    assert (w >= 1).all()
    s2, d2, w2 = oracle.sbm_sample(block, theta, om, 11)
    assert np.array_equal(s, s2) and np.array_equal(d, d2) and np.array_equal(w, w2)
    s3, _, _ = oracle.sbm_sample(block, theta, om, 12)
    assert not (len(s3) == len(s) and np.array_equal(s3, s))


def test_closed_forms():
    n = 7
    s, _, _ = oracle.sbm_sample(BLOCK7, THETA7, np.zeros((3, 3)), 1)
    assert len(s) == 0
    s, d, _ = oracle.sbm_sample(BLOCK7, THETA7, np.full((3, 3), 100.0), 1)   # every lambda >= 9
    assert sorted(zip(np.minimum(s, d).tolist(), np.maximum(s, d).tolist())) == \
        [(i, j) for i in range(n) for j in range(i + 1, n)]
    # one block: the upper triangle of one table
    s, d, _ = oracle.sbm_sample(np.zeros(5, np.int32), np.ones(5), np.full((1, 1), 100.0), 2)
    assert len(s) == 10 and (s < d).all()


def test_segmented_tables_have_the_expected_count_and_spread():
    # blocks of 300 and 400 nodes: tables of 44,850 (one segment), 120,000 and 79,800 entries
    # (two segments each)
    rng = np.random.default_rng(5)
    block = np.concatenate([np.zeros(300, np.int32), np.ones(400, np.int32)])
    rng.shuffle(block)
    theta = rng.uniform(0.5, 1.5, 700)
    om = np.array([[0.004, 0.001], [0.001, 0.003]])
    lam = _lam(block, theta, om)
    iu = np.triu_indices(700, 1)
    p = 1 - np.exp(-lam[iu])
    S = 300
    counts = np.zeros(S)
    # spread: nonzero entries by the first endpoint's decile of node index
    dec = np.zeros(10)
    for seed in range(S):
        s, d, _ = oracle.sbm_sample(block, theta, om, seed)
        counts[seed] = len(s)
        np.add.at(dec, np.minimum(s, d) * 10 // 700, 1)
    z = (counts.mean() - p.sum()) / np.sqrt((p * (1 - p)).sum() / S)
    assert abs(z) < 4.5, z
    exp_dec = np.zeros(10)
    np.add.at(exp_dec, iu[0] * 10 // 700, p)
    var_dec = np.zeros(10)
    np.add.at(var_dec, iu[0] * 10 // 700, p * (1 - p))
    zd = (dec / S - exp_dec) / np.sqrt(var_dec / S)
    assert np.abs(zd).max() < 4.5, zd
