"""bench.py's roofline arithmetic on CPU: the algorithmic work of a kernel family and the
achieved rate = work per launch / average launch duration, as a fraction of the peak."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


class _Graph:
    n = 1000
    nnz = 20000


WL = {"dims": (128, 128, 64), "kmax": 40}


def test_assign_work_counts_real_centroids_and_passes():
    cands = [(10, 0.5, 0.1, 7), (30, 0.4, 0.2, 3)]   # (K, modularity, NCut, passes)
    # the tensor-core family runs passes 2..p (pass 1 is its own family)
    bound, work, unit = bench.algorithmic_work("assign_tc", _Graph, WL, 2, cands)
    assert (bound, unit) == ("tensor", "FLOP")
    assert work == 2 * 64 * (1000 * 10 * 6 + 1000 * 30 * 2)
    # the FP32 family runs every pass
    bound, work_f, _ = bench.algorithmic_work("assign_ffma", _Graph, WL, 4, cands)
    assert bound == "alu" and work_f == 2 * 64 * (1000 * 10 * 7 + 1000 * 30 * 3)


def test_equal_nmi_rule_needs_both_clauses():
    q = {"nmi_planted": 0.745, "oracle": {"bf16_rounded_z": {"nmi_vs_oracle": 0.86}}}
    ok = bench.equal_nmi_rule(q, {"nmi_planted": 0.7447, "nmi_bf16_vs_fp32": 0.861})
    assert ok["equal_nmi"] and ok["equal_nmi_planted"] and ok["equal_nmi_agreement"]
    worse = bench.equal_nmi_rule(q, {"nmi_planted": 0.76, "nmi_bf16_vs_fp32": 0.861})
    assert not worse["equal_nmi"] and not worse["equal_nmi_planted"]
    apart = bench.equal_nmi_rule(q, {"nmi_planted": 0.745, "nmi_bf16_vs_fp32": 0.80})
    assert not apart["equal_nmi"] and not apart["equal_nmi_agreement"]


def test_seeding_work_is_one_plain_pass_per_round():
    bound, work, unit = bench.algorithmic_work("seed_update", _Graph, WL, 2, [])
    assert (bound, unit) == ("hbm", "B")
    assert work == 39 * 1000 * (64 * 2 + 8)


def test_roofline_fraction_is_work_per_launch_over_the_average_launch():
    cands = [(10, 0.0, 0.0, 5)]
    full = {"assign_tc": {"ms": 3.0, "launches": 5, "timed": 5}, "other": {"ms": 1.0, "launches": 2, "timed": 2}}
    # two timed steps of five launches, 2 ms each
    timed = {"assign_tc": {"ms": 20.0, "launches": 10, "timed": 10}}
    r = bench.roofline(full, timed, "assign_tc", _Graph, WL, 2, cands, steps=2)
    per_launch = 2 * 64 * 1000 * 10 * 4 / 5          # passes 2..5 of the candidate over 5 launches
    assert r["avg_launch_ms"] == pytest.approx(2.0)
    assert r["launches_per_step"] == 5
    assert r["achieved"] == pytest.approx(per_launch / 2e-3 / 1e12)
    assert r["unit"] == "TFLOP/s" and r["bound"] == "tensor"
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["shares"] == {"assign_tc": 0.75, "other": 0.25}
