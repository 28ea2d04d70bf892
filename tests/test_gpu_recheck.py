"""Near-tie re-check of the reported k-means labels (Section III-C, "apply KMeans").

With recheck = FP64 every reported label must equal the FP64 oracle's label bit for bit for
the same stored Z and the same centroids: the oracle's Lloyd with T = 1 assigns every point to
the argmin of the FP64 direct-form distance (ties to the lowest index).  The inputs hold
adversarial near ties: for a point z and a direction v orthogonal to it, a centroid mu_a and
its mirror image mu_b across the hyperplane through 0 and z (v^T x = 0) are exactly as far
from z and exactly as long, so after FP32 rounding of the centroids their distances differ by
about 1e-7, far inside every engine's error band.

Without a re-check, every label that differs from the FP64 argmin must differ by less than
twice the engine's derived score error (the band's model); that checks the model on the
hardware."""
import numpy as np
import pytest
import torch

import oracle
from paper_2312_01560_gb300 import api

pytestmark = pytest.mark.gpu


def _inputs(d, n=5003, pairs=150, k_rand=100, seed=0):
    rng = np.random.default_rng(seed + d)
    z = rng.normal(size=(n, d))
    z /= np.linalg.norm(z, axis=1, keepdims=True)
    zb = torch.tensor(z, dtype=torch.bfloat16).float().numpy().astype(np.float64)   # BF16-representable rows
    zb /= np.maximum(np.linalg.norm(zb, axis=1, keepdims=True), 1.0)                  # keep norms <= 1
    zb = torch.tensor(zb, dtype=torch.bfloat16).float().numpy().astype(np.float64)
    mus = []
    for t in range(pairs):
        p = zb[t]
        v = rng.normal(size=d)
        v -= (v @ p) / (p @ p) * p           # v orthogonal to z
        v /= np.linalg.norm(v)
        r = rng.normal(size=d)
        a = p + 0.3 * r / np.linalg.norm(r)
        a *= 0.95 / np.linalg.norm(a)
        b = a - 2.0 * (a @ v) * v             # mirror image: |b| = |a|, |b - z| = |a - z|
        mus += [a, b]
    r = rng.normal(size=(k_rand, d))
    mus += list(0.9 * r / np.linalg.norm(r, axis=1, keepdims=True))
    mu = np.array(mus, dtype=np.float32)
    return zb, mu


def _fp64_labels(Z, mu):
    lab, _, _ = oracle.lloyd(Z.astype(np.float64), mu.astype(np.float64), 1)
    return lab


def _band_model(engine, d):
    u = 2.0 ** -24
    if engine == "ffma":
        E = 3 * d * u * (1 + d * u) + 4 * u
    else:
        E = 2 * (2.0 ** -16 + (d / 8) * 17 * 2 * u * 1.01) + 1.01 * d * u + 13 * u
    return 2 * E


CASES = [("ffma", torch.float32), ("ffma", torch.bfloat16), ("tc", torch.bfloat16), ("tc8", torch.bfloat16)]


@pytest.mark.parametrize("engine,zdtype", CASES)
@pytest.mark.parametrize("d", [32, 64, 128])
def test_fp64_recheck_labels_are_the_oracle_labels(cuda, engine, zdtype, d):
    Z, mu = _inputs(d)
    ref = _fp64_labels(Z, mu)
    Zt = torch.tensor(Z, dtype=zdtype, device=cuda)
    lab, _, _ = api.lloyd(Zt, torch.tensor(mu, device=cuda), iters=1, assign=engine, recheck="fp64")
    lab = lab.cpu().numpy()
    assert np.array_equal(lab, ref), int((lab != ref).sum())


@pytest.mark.parametrize("engine,zdtype", CASES)
@pytest.mark.parametrize("d", [32, 64])
def test_fp64_recheck_after_lloyd_passes(cuda, engine, zdtype, d):
    # after several passes the reported labels are the FP64 argmin against the returned centroids
    Z, mu = _inputs(d, seed=7)
    Zt = torch.tensor(Z, dtype=zdtype, device=cuda)
    lab, mu_out, passes = api.lloyd(Zt, torch.tensor(mu, device=cuda), iters=6, assign=engine, recheck="fp64")
    ref = _fp64_labels(Z, mu_out.cpu().numpy())
    assert np.array_equal(lab.cpu().numpy(), ref)


@pytest.mark.parametrize("engine,zdtype", CASES)
@pytest.mark.parametrize("d", [32, 64, 128])
def test_unchecked_label_errors_stay_inside_the_band_model(cuda, engine, zdtype, d):
    Z, mu = _inputs(d, seed=3)
    ref = _fp64_labels(Z, mu)
    Zt = torch.tensor(Z, dtype=zdtype, device=cuda)
    mode = "none" if engine != "ffma" else "fp32"     # the FP32 engine's passes never re-check
    lab, _, _ = api.lloyd(Zt, torch.tensor(mu, device=cuda), iters=1, assign=engine, recheck=mode)
    lab = lab.cpu().numpy()
    bad = np.nonzero(lab != ref)[0]
    m64 = mu.astype(np.float64)
    gaps = [((Z[i] - m64[lab[i]]) ** 2).sum() - ((Z[i] - m64[ref[i]]) ** 2).sum() for i in bad]
    worst = max(gaps) if gaps else 0.0
    print(f"{engine} d={d}: {len(bad)} labels differ from the FP64 argmin without a re-check; "
          f"largest distance gap {worst:.3e}, band model {_band_model(engine, d):.3e}")
    assert worst <= _band_model(engine, d)


def test_select_with_fp64_recheck(cuda):
    from inputs.dcsbm import workload
    g = workload("dcsbm-1k")
    _, Z = oracle.embed(g, "mod_full", (64, 64, 64), seed=1)
    dg = api.DeviceGraph.from_host(g, cuda)
    Zt = torch.tensor(Z, dtype=torch.bfloat16, device=cuda)
    l1, r1 = api.select(dg, Zt, kmin=2, kmax=30, assign="tc", recheck="fp64")
    l2, r2 = api.select(dg, Zt, kmin=2, kmax=30, assign="tc", recheck="fp32")
    assert [c[0] for c in r1["cands"]] == [c[0] for c in r2["cands"]]
    lab = l1.cpu().numpy()
    _, _, mod, _ = oracle.score(g, lab, int(lab.max()) + 1)
    assert [c[1] for c in r1["cands"] if c[0] == r1["k"]][0] == mod
