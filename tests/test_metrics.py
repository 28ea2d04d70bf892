"""Partition-agreement metrics against hand values and (where installed) scikit-learn."""
import numpy as np
import pytest

from paper_2312_01560_gb300.metrics import ari, nmi


def test_identical_and_relabelled():
    a = np.array([0, 0, 1, 1, 2, 2])
    assert nmi(a, a) == 1.0 and ari(a, a) == 1.0
    assert nmi(a, 5 - a) == pytest.approx(1.0) and ari(a, 5 - a) == pytest.approx(1.0)


def test_hand_values():
    # one block vs two halves: H(U)=0, H(V)=ln 2, I=0 -> NMI 0; ARI 0
    a = np.zeros(4, int)
    b = np.array([0, 0, 1, 1])
    assert nmi(a, b) == 0.0
    assert ari(a, b) == 0.0


def test_against_sklearn():
    sk = pytest.importorskip("sklearn.metrics")
    rng = np.random.default_rng(0)
    for _ in range(5):
        a = rng.integers(0, 7, 500)
        b = np.where(rng.random(500) < 0.7, a, rng.integers(0, 9, 500))
        assert nmi(a, b) == pytest.approx(sk.normalized_mutual_info_score(a, b, average_method="arithmetic"), abs=1e-12)
        assert ari(a, b) == pytest.approx(sk.adjusted_rand_score(a, b), abs=1e-12)
