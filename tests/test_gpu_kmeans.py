"""GPU k-means steps against the oracle: k-means++ seeds bit-exact when both sides take the
D^2 decision in FP32 (same inputs); Lloyd labels equal where the nearest centroid is
unambiguous and valid (within the FP32 error bound) everywhere; centroids equal the FP64
means of their points; the empty-cluster and duplicate-point rules."""
import numpy as np
import pytest
import torch

import oracle
from inputs.dcsbm import workload
from paper_2312_01560_gb300 import api

pytestmark = pytest.mark.gpu


def _unit_rows(rng, n, d):
    z = rng.normal(size=(n, d))
    return z / np.linalg.norm(z, axis=1, keepdims=True)


@pytest.fixture(scope="module")
def z1k():
    g = workload("dcsbm-1k")
    _, Z = oracle.embed(g, "ncut", (64, 64, 32), seed=1)
    return Z.astype(np.float32)


@pytest.mark.parametrize("K", [1, 2, 40, 333])
def test_kmeanspp_bit_exact(cuda, z1k, K):
    seeds = api.kmeanspp(torch.tensor(z1k, device=cuda), K, seed=7).cpu().numpy()
    ref = oracle.kmeanspp(z1k.astype(np.float64), K, 7, fp32_decision=True)
    assert np.array_equal(seeds, ref)


@pytest.mark.parametrize("d", [32, 64, 128])
def test_kmeanspp_bit_exact_bf16_and_widths(cuda, d):
    rng = np.random.default_rng(d)
    Z = torch.tensor(_unit_rows(rng, 3001, d), dtype=torch.bfloat16, device=cuda)
    seeds = api.kmeanspp(Z, 64, seed=3).cpu().numpy()
    ref = oracle.kmeanspp(Z.float().cpu().numpy().astype(np.float64), 64, 3, fp32_decision=True)
    assert np.array_equal(seeds, ref)


def _clustered_rows(rng, n, d, k, spread):
    centres = _unit_rows(rng, k, d)
    z = centres[rng.integers(0, k, n)] + spread * rng.normal(size=(n, d)) / np.sqrt(d)
    return z / np.linalg.norm(z, axis=1, keepdims=True)


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float32])
def test_kmeanspp_bit_exact_many_blocks(cuda, dtype):
    # clustered rows, so the skip bound and the partial-row cut both fire; the point count
    # spreads ragged ranges over every SM's block
    rng = np.random.default_rng(11)
    Z = torch.tensor(_clustered_rows(rng, 150_001, 64, 300, 0.6), dtype=dtype, device=cuda)
    seeds = api.kmeanspp(Z, 200, seed=5).cpu().numpy()
    ref = oracle.kmeanspp(Z.float().cpu().numpy().astype(np.float64), 200, 5, fp32_decision=True)
    assert np.array_equal(seeds, ref)


def test_kmeanspp_bit_exact_chunked_row_lists(cuda):
    # 700 seed rows of 128 BF16 coordinates leave the persistent kernel room for one 32-row
    # group per warp list, so every warp reads its rows in two chunks per round
    rng = np.random.default_rng(14)
    Z = torch.tensor(_clustered_rows(rng, 300_007, 128, 60, 0.6), dtype=torch.bfloat16, device=cuda)
    seeds = api.kmeanspp(Z, 700, seed=6).cpu().numpy()
    ref = oracle.kmeanspp(Z.float().cpu().numpy().astype(np.float64), 700, 6, fp32_decision=True)
    assert np.array_equal(seeds, ref)


def test_kmeanspp_bit_exact_per_round_kernels(cuda):
    # 450 seed rows of 128 FP32 coordinates do not fit the persistent kernel's shared memory,
    # so the seeding runs as one update and one pick launch per round
    rng = np.random.default_rng(12)
    Z = torch.tensor(_clustered_rows(rng, 4000, 128, 50, 0.5), dtype=torch.float32, device=cuda)
    seeds = api.kmeanspp(Z, 450, seed=2).cpu().numpy()
    ref = oracle.kmeanspp(Z.cpu().numpy().astype(np.float64), 450, 2, fp32_decision=True)
    assert np.array_equal(seeds, ref)


def test_kmeanspp_duplicates(cuda):
    Z = torch.zeros((50, 32), device=cuda)
    Z[:, 0] = 1.0
    Z[40:, 0] = 0.0
    Z[40:, 1] = 1.0                  # two distinct points, 40 + 10 copies
    seeds = api.kmeanspp(Z, 6, seed=1).cpu().numpy()
    assert np.array_equal(seeds, oracle.kmeanspp(Z.cpu().numpy().astype(np.float64), 6, 1, fp32_decision=True))
    assert len(set(seeds.tolist())) == 6


def _validate(Z, labels, mu, tol=2e-5):
    Z = Z.astype(np.float64)
    d2 = ((Z[:, None, :] - mu[None, :, :].astype(np.float64)) ** 2).sum(-1)
    chosen = d2[np.arange(Z.shape[0]), labels]
    assert (chosen <= d2.min(axis=1) + tol).all()


def test_lloyd_matches_oracle_on_separated_blobs(cuda):
    rng = np.random.default_rng(3)
    centres = _unit_rows(rng, 12, 64)
    lab_true = rng.integers(0, 12, 4000)
    Z = centres[lab_true] + 0.05 * rng.normal(size=(4000, 64))
    Z = (Z / np.linalg.norm(Z, axis=1, keepdims=True)).astype(np.float32)
    mu0 = Z[rng.choice(4000, 12, replace=False)]
    lab, mu, passes = api.lloyd(torch.tensor(Z, device=cuda), torch.tensor(mu0, device=cuda), iters=50)
    lo, muo, po = oracle.lloyd(Z.astype(np.float64), mu0.astype(np.float64), 50)
    assert np.array_equal(lab.cpu().numpy(), lo) and passes == po
    np.testing.assert_allclose(mu.cpu().numpy(), muo, atol=1e-6)


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_lloyd_generic_embeddings(cuda, z1k, dtype):
    Zt = torch.tensor(z1k, device=cuda).to(dtype)
    Z = Zt.float().cpu().numpy()
    seeds = oracle.kmeanspp(Z.astype(np.float64), 30, 5, fp32_decision=True)
    mu0 = Z[seeds]
    lab, mu, passes = api.lloyd(Zt, torch.tensor(mu0, device=cuda), iters=50)
    lab = lab.cpu().numpy()
    mu = mu.cpu().numpy()
    lo, muo, po = oracle.lloyd(Z.astype(np.float64), mu0.astype(np.float64), 50)
    assert (lab == lo).mean() >= 0.995
    if passes < 50:                                  # converged: labels are a fixed point
        _validate(Z, lab, mu)
        for c in np.unique(lab):
            np.testing.assert_allclose(mu[c], Z[lab == c].astype(np.float64).mean(0), atol=2e-7)


def test_lloyd_empty_cluster_keeps_centroid(cuda):
    Z = np.zeros((6, 32), np.float32)
    Z[:3, 0] = 1.0
    Z[3:, 1] = 1.0
    mu0 = np.zeros((3, 32), np.float32)
    mu0[0, 0] = 0.9
    mu0[1, 1] = 0.9
    mu0[2, 2] = -1.0                     # never the nearest
    lab, mu, _ = api.lloyd(torch.tensor(Z, device=cuda), torch.tensor(mu0, device=cuda), iters=10)
    assert lab.cpu().tolist() == [0, 0, 0, 1, 1, 1]
    assert mu[2, 2].item() == -1.0 and mu[0, 0].item() == 1.0


def test_lloyd_k_equals_n(cuda):
    rng = np.random.default_rng(9)
    Z = _unit_rows(rng, 100, 32).astype(np.float32)
    lab, _, passes = api.lloyd(torch.tensor(Z, device=cuda), torch.tensor(Z, device=cuda), iters=5)
    assert lab.cpu().tolist() == list(range(100)) and passes == 2


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float32])
def test_kmeanspp_16_byte_aligned_rows(cuda, dtype):
    # Z starting 16 bytes past a 32-byte boundary takes the 16-byte loads of the seeding
    # update instead of the 32-byte ones: the same seeds
    rng = np.random.default_rng(13)
    host = torch.tensor(_clustered_rows(rng, 20_003, 64, 40, 0.6), dtype=dtype)
    esz = host.element_size()
    raw = torch.zeros(host.numel() * esz + 64, dtype=torch.uint8, device=cuda)
    Z = raw[16:16 + host.numel() * esz].view(dtype).view(host.shape)
    Z.copy_(host.to(cuda))
    assert Z.data_ptr() % 32 == 16
    seeds = api.kmeanspp(Z, 120, seed=4).cpu().numpy()
    ref = oracle.kmeanspp(host.float().numpy().astype(np.float64), 120, 4, fp32_decision=True)
    assert np.array_equal(seeds, ref)


def test_misaligned_z_is_rejected(cuda):
    raw = torch.zeros(64 * 32 * 4 + 64, dtype=torch.uint8, device=cuda)
    Z = raw[8:8 + 64 * 32 * 4].view(torch.float32).view(64, 32)
    assert Z.data_ptr() % 16 == 8
    with pytest.raises(RuntimeError, match="16-byte aligned"):
        api.kmeanspp(Z, 4, seed=1)
    mu0 = torch.zeros(4, 32)
    with pytest.raises(RuntimeError, match="16-byte aligned"):
        api.lloyd(Z, mu0, iters=2)
