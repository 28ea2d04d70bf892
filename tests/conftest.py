import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built CUDA library")


import pytest  # noqa: E402


@pytest.fixture(scope="session")
def cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_01560_gb300 import _abi
    _abi.lib()          # the CUDA library must be built; no fallback
    return torch.device("cuda:0")


def rel_fro(a, b):
    import numpy as np
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def ragged_graph(seed=0):
    """Isolated nodes, a hub row longer than a warp's column chunk, N not a tile multiple."""
    import numpy as np
    from inputs.dcsbm import from_edges
    rng = np.random.default_rng(seed)
    n = 1237
    m = 6000
    u = rng.integers(0, n - 7, m)
    v = rng.integers(0, n - 7, m)
    hub_u = np.zeros(700, np.int64) + 3
    hub_v = rng.choice(np.arange(10, n - 7), 700, replace=False)
    return from_edges(n, np.concatenate([u, hub_u]), np.concatenate([v, hub_v]))
