"""The N > 1 path of bench.py, on CPU: the method does not shard (one graph per GPU), so
`bench.py --gpus N` runs N independent replicas and reports their whole-job rate, N graphs
over the slowest rank's time.  Here two ranks on a gloo process group check that aggregation,
and that the oracle arm runs on rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _replica(rank, world, port, ms_local, units, queue):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    value, ms = bench.replica_throughput(ms_local, units, world)
    queue.put((rank, value, ms))
    dist.destroy_process_group()


def test_replica_throughput_is_all_units_over_the_slowest_rank():
    world, units = 2, 11_597_080
    times = [40.0, 55.5]   # ms per step on each rank
    ctx = mp.get_context("spawn")
    queue = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_replica, args=(r, world, port, times[r], units, queue)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(queue.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    for rank, value, ms in got:
        assert ms == max(times)
        assert value == pytest.approx(world * units / (max(times) * 1e-3), rel=1e-12)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    value, ms = bench.replica_throughput(50.0, 1000, 1)
    assert (value, ms) == (pytest.approx(20_000.0), 50.0)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
