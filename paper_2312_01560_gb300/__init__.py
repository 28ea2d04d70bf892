"""RaftGP (random fast graph partitioning) hot path for GB300 (sm_103a).

Stages (Section III of the paper): Gaussian random projection of the NCut / modularity
operators (Eq. 5), a randomly initialised GCN (Eq. 6) with row l2-normalisation, and model
selection over candidate K by k-means scored with modularity (Eq. 3) or NCut (Eq. 1).
All compute runs in libraftgp.so (hand-written CUDA for sm_103a) behind the C ABI of
include/raftgp.h; this package marshals torch tensors into it.
"""
from .metrics import ari, nmi  # noqa: F401

__all__ = ["DeviceGraph", "embed", "select", "partition", "score", "kmeanspp", "lloyd", "version", "nmi", "ari"]


def __getattr__(name):
    if name in ("DeviceGraph", "embed", "select", "partition", "score", "kmeanspp", "lloyd", "version",
                "workspace_size", "embed_opts", "select_opts"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
