"""Write the FP64 oracle's partitions of the 50,000- and 1,000,000-node workloads.

Calls only the oracle (``oracle/``) and the seeded input generator (``inputs/``); nothing
here touches the CUDA library.  Each output file holds, for one workload:
  - ``labels``: the oracle's chosen partition (Section III-C model selection on the FP64
    embedding of Eq. 5 and Eq. 6);
  - ``labels_z32``: the oracle's partition of the same embedding rounded once to FP32 (the
    sensitivity of the k-means model selection to one single-precision rounding of Z);
  - ``labels_zbf16`` (1M-node workload): the same with Z rounded once to BF16 (round to nearest
    even), the perturbation BF16 storage of the final embedding alone brings;
  - ``cands`` / ``cands_z32`` / ``cands_zbf16``: (K, Mod, NCut, Lloyd passes) per evaluated
    candidate, and ``k`` / ``k_z32`` / ``k_zbf16`` the chosen K;
  - ``fingerprint``: SHA-256 of the graph's CSR (``inputs.dcsbm.fingerprint``), so a reader
    checks that its graph is the one these labels belong to;
  - the configuration (operator, layer widths, K range, grid, pass cap, seeds).
A second file per workload, ``oracle_stages_<name>.npz``, holds the oracle's values of every
embedding stage (Y of Eq. 5, then Z^(1..n) of Eq. 6 with the row normalisation) on 64 seeded
sample rows (63 uniform and the highest-degree node), for per-stage error reports.

  python tests/golden/make_oracle_partitions.py [dcsbm-50k] [dcsbm-1m] [--threads T] [--stages-only]

The 1,000,000-node run takes about an hour of CPU time on 8 cores (about 3e13 FP64
operations in the k-means passes)."""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from inputs.dcsbm import fingerprint, workload  # noqa: E402

# Embedding seed 1, selection seed 2; the modularity operator applied as a sparse product plus
# a rank-one term; ten coarse and ten refined candidates; at most 50 Lloyd passes.
CONFIGS = {
    "dcsbm-50k": dict(op="mod_full", dims=(128, 128, 64), kmin=2, kmax=100, grid=10, T=50,
                      embed_seed=1, select_seed=2),
    "dcsbm-1m": dict(op="mod_full", dims=(128, 128, 128, 128, 64), kmin=50, kmax=400, grid=10, T=50,
                     embed_seed=1, select_seed=2),
}


def path_for(name: str) -> str:
    return os.path.join(HERE, f"oracle_partition_{name}.npz")


def stages_path_for(name: str) -> str:
    return os.path.join(HERE, f"oracle_stages_{name}.npz")


def load_stages(name: str) -> dict:
    """rows (int64), stage0 .. stageL (FP64, one row per sample), fingerprint, config."""
    with np.load(stages_path_for(name)) as f:
        out = {k: f[k] for k in f.files}
    out["fingerprint"] = str(out["fingerprint"])
    out["config"] = json.loads(str(out["config"]))
    return out


def make_stages(name: str, n_rows: int = 64) -> None:
    cfg = CONFIGS[name]
    g = workload(name)
    dims, seed = cfg["dims"], cfg["embed_seed"]
    rng = np.random.default_rng(12345)
    rows = np.sort(np.concatenate([rng.choice(g.n, n_rows - 1, replace=False), [int(np.argmax(g.degrees()))]]))
    rows = np.unique(rows).astype(np.int64)
    t0 = time.time()
    theta = oracle.theta(g.n, dims[0], seed)
    Y = oracle.project(g, cfg["op"], theta)
    del theta
    out = {"stage0": Y[rows]}
    Zk = Y
    for k in range(1, len(dims)):
        Zk = oracle.gcn_layer(g, Zk, oracle.gcn_weight(k, dims[k - 1], dims[k], seed))
        out[f"stage{k}"] = Zk[rows]
    # the stage-by-stage chain is the oracle's whole embedding
    _, Z = oracle.embed(g, cfg["op"], dims, seed)
    assert np.array_equal(Z[rows], out[f"stage{len(dims) - 1}"])
    np.savez_compressed(stages_path_for(name), rows=rows, fingerprint=np.str_(fingerprint(g)),
                        config=np.str_(json.dumps(cfg)), **out)
    print(f"{name}: stage rows in {time.time() - t0:.1f} s, wrote {stages_path_for(name)}", flush=True)


def load(name: str) -> dict:
    """The stored partition of workload `name` as a dict (labels, labels_z32, k, k_z32, cands,
    cands_z32, fingerprint, config)."""
    with np.load(path_for(name)) as f:
        out = {k: f[k] for k in f.files}
    for tag in VARIANTS:
        if "labels" + tag in out:
            out["labels" + tag] = out["labels" + tag].astype(np.int32)
            out["k" + tag] = int(out["k" + tag])
    out["fingerprint"] = str(out["fingerprint"])
    out["config"] = json.loads(str(out["config"]))
    return out


def round_bf16(x: np.ndarray) -> np.ndarray:
    """x rounded to the nearest BF16 value (ties to even), returned in FP64: the FP32 bits with
    the low 16 bits rounded away (inputs are finite)."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


VARIANTS = {"": lambda Z: Z, "_z32": lambda Z: Z.astype(np.float32).astype(np.float64), "_zbf16": round_bf16}


def make(name: str, variants=("", "_z32")) -> None:
    """Computes the listed variants (keeping the ones already stored for the same graph)."""
    cfg = CONFIGS[name]
    g = workload(name)
    fp = fingerprint(g)
    res = {}
    if os.path.exists(path_for(name)):
        with np.load(path_for(name)) as f:
            if str(f["fingerprint"]) == fp and json.loads(str(f["config"])) == json.loads(json.dumps(cfg)):
                res = {k: f[k] for k in f.files if k not in ("fingerprint", "config")}
    t0 = time.time()
    _, Z = oracle.embed(g, cfg["op"], cfg["dims"], cfg["embed_seed"])
    t1 = time.time()
    print(f"{name}: embedding {t1 - t0:.1f} s", flush=True)
    for tag in variants:
        r = oracle.select(g, VARIANTS[tag](Z), cfg["kmin"], cfg["kmax"], cfg["grid"], cfg["T"], cfg["select_seed"])
        res["labels" + tag] = r["labels"].astype(np.uint16)
        res["k" + tag] = np.int32(r["k"])
        res["cands" + tag] = np.array(r["cands"], dtype=np.float64)
        print(f"{name}{tag}: K* = {r['k']}, selection {time.time() - t1:.1f} s", flush=True)
        t1 = time.time()
        np.savez_compressed(path_for(name), fingerprint=np.str_(fp), config=np.str_(json.dumps(cfg)), **res)
    print(f"wrote {path_for(name)}", flush=True)


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("names", nargs="*", default=list(CONFIGS))
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--stages-only", action="store_true")
    ap.add_argument("--variants", default=None,
                    help="comma-separated subset of '', '_z32', '_zbf16' (default: all three for dcsbm-1m, "
                         "the first two otherwise)")
    a = ap.parse_args()
    print(f"oracle threads: {oracle.set_threads(a.threads)}", flush=True)
    for nm in a.names:
        if not a.variants:
            make_stages(nm)
        if not a.stages_only:
            vs = a.variants.split(",") if a.variants is not None else (
                ["", "_z32", "_zbf16"] if nm == "dcsbm-1m" else ["", "_z32"])
            make(nm, [("" if v in ("''", '""', "base") else v) for v in vs])
