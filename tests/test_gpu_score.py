"""GPU partition scoring against the oracle: block edge counts and volumes bit-exact
(int64), modularity (Eq. 3 via Eq. 7) and NCut (Eq. 1) bit-exact FP64."""
import numpy as np
import pytest
import torch

import oracle
from conftest import ragged_graph
from inputs import small
from inputs.dcsbm import workload
from paper_2312_01560_gb300 import api

pytestmark = pytest.mark.gpu


def _check(g, labels, K, dev, bits=None):
    dg = api.DeviceGraph.from_host(g, dev, row_ptr_bits=bits)
    m, vol, mod, ncut = api.score(dg, torch.tensor(labels, dtype=torch.int32, device=dev), K)
    mo, vo, modo, ncuto = oracle.score(g, labels, K)
    assert np.array_equal(m.cpu().numpy(), mo)
    assert np.array_equal(vol.cpu().numpy(), vo)
    assert mod == modo and ncut == ncuto        # bit-exact
    return mod, ncut


@pytest.mark.parametrize("K", [1, 2, 11, 97, 1000])
@pytest.mark.parametrize("bits", [32, 64])
def test_random_labels_bit_exact(cuda, K, bits):
    g = workload("dcsbm-1k")
    labels = np.random.default_rng(K).integers(0, K, g.n).astype(np.int32)
    _check(g, labels, K, cuda, bits)


def test_planted_and_ragged(cuda):
    g = workload("dcsbm-50k")
    _check(g, g.planted, g.k_planted, cuda)
    r = ragged_graph(2)
    _check(r, (np.arange(r.n) % 13).astype(np.int32), 13, cuda)


def test_ring_of_cliques_closed_form(cuda):
    g = small.ring_of_cliques(7, 6)
    mod, ncut = _check(g, g.planted, 7, cuda)
    mm = 15
    assert mod == pytest.approx(mm / (mm + 1) - 1 / 7, abs=1e-15)
    assert ncut == pytest.approx(7 / (2 * (mm + 1)), abs=1e-15)


def test_label_out_of_range_is_rejected(cuda):
    g = workload("dcsbm-1k")
    dg = api.DeviceGraph.from_host(g, cuda)
    lab = torch.zeros(g.n, dtype=torch.int32, device=cuda)
    lab[10] = 5
    with pytest.raises(api._abi.RaftgpError, match="EINVAL"):
        api.score(dg, lab, 3)


def test_full_size_bit_exact(cuda):
    g = workload("dcsbm-1m")
    labels = np.random.default_rng(0).integers(0, 400, g.n).astype(np.int32)
    _check(g, labels, 400, cuda, bits=64)
    _check(g, g.planted, g.k_planted, cuda, bits=64)
