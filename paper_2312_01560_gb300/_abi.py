"""ctypes mirror of include/raftgp.h and the loader of libraftgp.so.

The library is loaded from this package directory only; if it is missing the import of the
compute functions raises (there is no CPU fallback)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libraftgp.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EUNSUPPORTED = range(6)
STATUS_NAMES = {0: "RAFTGP_OK", 1: "RAFTGP_EINVAL", 2: "RAFTGP_ENOMEM", 3: "RAFTGP_ECUDA", 4: "RAFTGP_ETIMEOUT",
                5: "RAFTGP_EUNSUPPORTED"}
OP = {"ncut": 0, "mod_full": 1, "mod_reduced": 2}
DTYPE = {"f32": 0, "bf16": 1}
CRIT = {"mod": 0, "ncut": 1}
ASSIGN = {"ffma": 0, "tc": 1, "tc8": 2}
RECHECK = {"none": 0, "fp32": 1, "fp64": 2}
MAX_LAYERS = 4
MAX_BATCH_CAND = 64

# Every entry point declared in include/raftgp.h.
EXPORTS = ("raftgp_workspace_size", "raftgp_embed", "raftgp_select", "raftgp_partition", "raftgp_score",
           "raftgp_kmeanspp", "raftgp_kmeanspp_noalloc", "raftgp_lloyd", "raftgp_lloyd_workspace_size", "raftgp_profile_enable", "raftgp_profile_enable_family", "raftgp_profile_read", "raftgp_last_error", "raftgp_debug_seed_skip_block",
           "raftgp_version", "raftgp_diff_workspace_size", "raftgp_gcn_layer_forward", "raftgp_gcn_layer_backward",
           "raftgp_softmod_loss", "raftgp_centroids", "raftgp_gcn_weights", "raftgp_adam_step",
           "raftgp_diff_plan_create", "raftgp_diff_plan_layer_forward", "raftgp_diff_plan_layer_backward",
           "raftgp_diff_plan_softmod_loss", "raftgp_diff_plan_destroy",
           "raftgp_batch_workspace_size", "raftgp_batch_plan_create", "raftgp_batch_plan_run", "raftgp_batch_plan_embedding", "raftgp_batch_plan_check",
           "raftgp_batch_plan_tuning_embed",
           "raftgp_batch_plan_candidates", "raftgp_batch_plan_tuning", "raftgp_batch_plan_destroy",
           "raftgp_partition_batched", "raftgp_bisect_workspace_size", "raftgp_select_bisect",
           "raftgp_select_bisect_update",
           "raftgp_sbm_workspace_size", "raftgp_sbm_count", "raftgp_sbm_emit", "raftgp_coo_to_csr_workspace_size",
           "raftgp_coo_to_csr", "raftgp_stream_workspace_size", "raftgp_stream_create", "raftgp_stream_add_edges",
           "raftgp_stream_info", "raftgp_stream_copy", "raftgp_stream_destroy")
BATCH_SLOTS = 20


class Csr(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("row_ptr", C.c_void_p), ("row_ptr_bits", C.c_int32),
                ("col", C.c_void_p)]


class EmbedOpts(C.Structure):
    _fields_ = [("op", C.c_int32), ("n_layers", C.c_int32), ("dims", C.c_int32 * (MAX_LAYERS + 1)),
                ("dtype", C.c_int32), ("seed", C.c_uint64), ("theta", C.c_void_p),
                ("W", C.c_void_p * MAX_LAYERS), ("stage_out", C.c_void_p * (MAX_LAYERS + 1))]


class BisectOpts(C.Structure):
    _fields_ = [("eps", C.c_int32), ("iters", C.c_int32), ("reading", C.c_int32), ("seed", C.c_uint64)]


class Sbm(C.Structure):
    _fields_ = [("n", C.c_int64), ("k", C.c_int32), ("block", C.c_void_p), ("theta", C.c_void_p),
                ("omega", C.c_void_p), ("seed", C.c_uint64)]


class BatchOpts(C.Structure):
    _fields_ = [("kmin", C.c_int32), ("kmax_factor", C.c_float), ("grid", C.c_int32), ("iters", C.c_int32),
                ("criterion", C.c_int32), ("lloyd_variant", C.c_int32), ("embed_variant", C.c_int32),
                ("assign", C.c_int32),
                ("seed", C.c_uint64)]


class SelectOpts(C.Structure):
    _fields_ = [("kmin", C.c_int32), ("kmax", C.c_int32), ("grid", C.c_int32), ("iters", C.c_int32),
                ("criterion", C.c_int32), ("assign", C.c_int32), ("batch", C.c_int32), ("recheck", C.c_int32),
                ("seed", C.c_uint64)]


class SelectResult(C.Structure):
    _fields_ = [("k_best", C.c_int32), ("n_cand", C.c_int32), ("cand_cap", C.c_int32),
                ("cand_k", C.POINTER(C.c_int32)), ("cand_mod", C.POINTER(C.c_double)),
                ("cand_ncut", C.POINTER(C.c_double)), ("cand_passes", C.POINTER(C.c_int32))]


class ProfEntry(C.Structure):
    _fields_ = [("name", C.c_char_p), ("launches", C.c_int64), ("timed", C.c_int64), ("ms", C.c_double)]


class RaftgpError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None


def lib():
    """The loaded libraftgp.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libraftgp.so is not built ({LIB_PATH} missing): run "
                               "`python -c 'import __graft_entry__ as g; g.build()'` first")
        L = C.CDLL(LIB_PATH)
        P = C.c_void_p
        L.raftgp_workspace_size.restype = C.c_size_t
        L.raftgp_workspace_size.argtypes = [C.POINTER(Csr), C.POINTER(EmbedOpts), C.POINTER(SelectOpts), C.c_int32]
        L.raftgp_embed.argtypes = [C.POINTER(Csr), C.POINTER(EmbedOpts), P, P, C.c_size_t, P]
        L.raftgp_select.argtypes = [C.POINTER(Csr), P, C.c_int32, C.c_int32, C.POINTER(SelectOpts), P,
                                    C.POINTER(SelectResult), P, C.c_size_t, P]
        L.raftgp_partition.argtypes = [C.POINTER(Csr), C.POINTER(EmbedOpts), C.POINTER(SelectOpts), P,
                                       C.POINTER(SelectResult), P, C.c_size_t, P]
        L.raftgp_score.argtypes = [C.POINTER(Csr), P, C.c_int32, P, P, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                   P, C.c_size_t, P]
        L.raftgp_kmeanspp.argtypes = [P, C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_uint64, P, P, C.c_size_t, P]
        L.raftgp_kmeanspp_noalloc.argtypes = [P, C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_uint64, P, P]
        L.raftgp_kmeanspp_noalloc.restype = C.c_int
        L.raftgp_lloyd.argtypes = [P, C.c_int64, C.c_int32, C.c_int32, P, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                   P, P, C.POINTER(C.c_int32), P, C.c_size_t, P]
        for name in ("raftgp_embed", "raftgp_select", "raftgp_partition", "raftgp_score", "raftgp_kmeanspp",
                     "raftgp_lloyd"):
            getattr(L, name).restype = C.c_int
        L.raftgp_profile_enable.restype = C.c_int
        L.raftgp_profile_enable.argtypes = [C.c_int32]
        L.raftgp_debug_seed_skip_block.argtypes = [C.c_int32]
        L.raftgp_debug_seed_skip_block.restype = None
        L.raftgp_profile_enable_family.restype = C.c_int
        L.raftgp_profile_enable_family.argtypes = [C.c_char_p]
        L.raftgp_profile_read.restype = C.c_int32
        L.raftgp_profile_read.argtypes = [C.POINTER(ProfEntry), C.c_int32]
        L.raftgp_diff_workspace_size.restype = C.c_size_t
        L.raftgp_diff_workspace_size.argtypes = [C.c_int64, C.c_int32, C.c_int32]
        L.raftgp_gcn_layer_forward.argtypes = [C.POINTER(Csr), P, C.c_int32, P, C.c_int32, P, P, C.c_size_t, P]
        L.raftgp_gcn_layer_backward.argtypes = [C.POINTER(Csr), P, C.c_int32, P, C.c_int32, P, P, P, P, C.c_size_t, P]
        L.raftgp_softmod_loss.argtypes = [C.POINTER(Csr), P, C.c_int32, P, C.c_int32, C.c_float,
                                          C.POINTER(C.c_double), P, P, C.c_size_t, P]
        L.raftgp_centroids.argtypes = [P, C.c_int64, C.c_int32, P, C.c_int32, P, P, C.c_size_t, P]
        L.raftgp_adam_step.argtypes = [P, P, P, P, C.c_int64, C.c_float, C.c_float, C.c_float, C.c_float, C.c_int32,
                                       P]
        L.raftgp_gcn_weights.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_uint64, P, P]
        L.raftgp_diff_plan_create.argtypes = [C.POINTER(Csr), C.c_int32, C.c_int32, P, C.c_size_t, P,
                                              C.POINTER(C.c_void_p)]
        L.raftgp_diff_plan_layer_forward.argtypes = [C.c_void_p, P, C.c_int32, P, C.c_int32, P, P]
        L.raftgp_diff_plan_layer_backward.argtypes = [C.c_void_p, P, C.c_int32, P, C.c_int32, P, P, P, P]
        L.raftgp_diff_plan_softmod_loss.argtypes = [C.c_void_p, P, C.c_int32, P, C.c_int32, C.c_float, P, P, P]
        L.raftgp_diff_plan_destroy.argtypes = [C.c_void_p]
        L.raftgp_diff_plan_destroy.restype = None
        for name in ("raftgp_gcn_layer_forward", "raftgp_gcn_layer_backward", "raftgp_softmod_loss",
                     "raftgp_centroids", "raftgp_gcn_weights", "raftgp_adam_step", "raftgp_diff_plan_create",
                     "raftgp_diff_plan_layer_forward", "raftgp_diff_plan_layer_backward",
                     "raftgp_diff_plan_softmod_loss"):
            getattr(L, name).restype = C.c_int
        I64P = C.POINTER(C.c_int64)
        L.raftgp_batch_workspace_size.restype = C.c_size_t
        L.raftgp_batch_workspace_size.argtypes = [C.POINTER(Csr), I64P, C.c_int32, C.POINTER(EmbedOpts),
                                                  C.POINTER(BatchOpts)]
        L.raftgp_batch_plan_create.argtypes = [C.POINTER(Csr), I64P, C.c_int32, C.POINTER(EmbedOpts),
                                               C.POINTER(BatchOpts), P, P, P, C.c_size_t, P, C.POINTER(C.c_void_p)]
        L.raftgp_batch_plan_run.argtypes = [C.c_void_p, P]
        L.raftgp_batch_plan_embedding.argtypes = [C.c_void_p, P]
        L.raftgp_batch_plan_check.argtypes = [C.c_void_p]
        L.raftgp_batch_plan_tuning_embed.argtypes = [C.c_void_p, C.POINTER(C.c_int32), P]
        L.raftgp_batch_plan_tuning_embed.restype = C.c_int
        L.raftgp_batch_plan_candidates.argtypes = [C.c_void_p, P, P, P, P]
        L.raftgp_batch_plan_tuning.argtypes = [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                               C.POINTER(C.c_float)]
        L.raftgp_batch_plan_destroy.argtypes = [C.c_void_p]
        L.raftgp_batch_plan_destroy.restype = None
        L.raftgp_partition_batched.argtypes = [C.POINTER(Csr), I64P, C.c_int32, C.POINTER(EmbedOpts),
                                               C.POINTER(BatchOpts), P, P, P, C.c_size_t, P]
        for name in ("raftgp_batch_plan_create", "raftgp_batch_plan_run", "raftgp_batch_plan_candidates",
                     "raftgp_batch_plan_tuning", "raftgp_batch_plan_embedding", "raftgp_batch_plan_check",
                     "raftgp_partition_batched"):
            getattr(L, name).restype = C.c_int
        L.raftgp_bisect_workspace_size.restype = C.c_size_t
        L.raftgp_bisect_workspace_size.argtypes = [C.c_int64, C.c_int32, C.c_int32]
        L.raftgp_select_bisect.restype = C.c_int
        L.raftgp_select_bisect.argtypes = [C.POINTER(Csr), P, C.c_int32, C.c_int32, C.POINTER(BisectOpts), P, P,
                                           C.POINTER(C.c_int32), P, C.c_size_t, P]
        L.raftgp_select_bisect_update.restype = C.c_int
        L.raftgp_select_bisect_update.argtypes = [C.POINTER(Csr), P, C.c_int32, C.c_int32, C.POINTER(BisectOpts), P,
                                                  C.c_int32, P, P, P, P, C.POINTER(C.c_int32), P, C.c_size_t, P]
        L.raftgp_lloyd_workspace_size.restype = C.c_size_t
        L.raftgp_lloyd_workspace_size.argtypes = [C.c_int64, C.c_int32, C.c_int32]
        L.raftgp_sbm_workspace_size.restype = C.c_size_t
        L.raftgp_sbm_workspace_size.argtypes = [C.c_int64, C.c_int32]
        L.raftgp_sbm_count.restype = C.c_int
        L.raftgp_sbm_count.argtypes = [C.POINTER(Sbm), C.POINTER(C.c_int64), P, C.c_size_t, P]
        L.raftgp_sbm_emit.restype = C.c_int
        L.raftgp_sbm_emit.argtypes = [C.POINTER(Sbm), P, P, P, C.c_int64, P, C.c_size_t, P]
        L.raftgp_coo_to_csr_workspace_size.restype = C.c_size_t
        L.raftgp_coo_to_csr_workspace_size.argtypes = [C.c_int64]
        L.raftgp_coo_to_csr.restype = C.c_int
        L.raftgp_coo_to_csr.argtypes = [C.c_int64, C.c_int64, P, P, P, P, P, C.c_size_t, P]
        L.raftgp_stream_workspace_size.restype = C.c_size_t
        L.raftgp_stream_workspace_size.argtypes = [C.c_int64, C.c_int64, C.POINTER(EmbedOpts)]
        L.raftgp_stream_create.restype = C.c_int
        L.raftgp_stream_create.argtypes = [C.POINTER(Csr), C.POINTER(EmbedOpts), C.c_int64, P, C.c_size_t,
                                           C.POINTER(P), P]
        L.raftgp_stream_add_edges.restype = C.c_int
        L.raftgp_stream_add_edges.argtypes = [P, P, P, C.c_int64, P]
        L.raftgp_stream_info.restype = C.c_int
        L.raftgp_stream_info.argtypes = [P, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        L.raftgp_stream_copy.restype = C.c_int
        L.raftgp_stream_copy.argtypes = [P, P, P, P, P]
        L.raftgp_stream_destroy.restype = None
        L.raftgp_stream_destroy.argtypes = [P]
        L.raftgp_last_error.restype = C.c_char_p
        L.raftgp_last_error.argtypes = []
        L.raftgp_version.restype = C.c_char_p
        L.raftgp_version.argtypes = []
        _lib = L
    return _lib


def check(status):
    if status != OK:
        raise RaftgpError(status, lib().raftgp_last_error().decode())
