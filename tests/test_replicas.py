"""The N > 1 path on CPU: ranks are independent replicas of the workload (no data-path
collective); the only cross-rank steps are the barrier and the max over ranks of the timed
region.  Two gloo ranks on 127.0.0.1 exercise both, and torchrun runs the reference arm of
bench.py with two ranks (rank 0 prints the one JSON line, rank 1 exits 0 without work)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        got = bench.max_over_ranks(10.0 * rank + 1.5, world, torch.device("cpu"))
        seeds = bench.replica_seeds(rank, 3)
        dist.barrier()
        q.put((rank, got, seeds))
    finally:
        dist.destroy_process_group()


def test_replica_seeds_disjoint():
    import bench
    world, B = 4, 5
    allseeds = [s for r in range(world) for s in bench.replica_seeds(r, B)]
    assert sorted(allseeds) == list(range(world * B))
    assert bench.replica_seeds(0, 2) == [0, 1]


def test_max_over_ranks_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(3.25, 1, None) == 3.25


def test_max_over_ranks_gloo_two_ranks():
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = {}
    try:
        for _ in range(world):
            rank, got, seeds = q.get(timeout=120)
            out[rank] = (got, seeds)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    # every rank sees the slowest rank's time
    assert out[0][0] == out[1][0] == 11.5
    assert set(out[0][1]).isdisjoint(out[1][1])


@pytest.mark.timeout(600)
def test_reference_arm_under_torchrun_two_ranks():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--workload", "deblur64_fp64", "--steps", "1", "--warmup", "0"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    p = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=540)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, p.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2
    assert d["value"] > 0 and d["unit"] == "solves/s"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"


def _rank_leaves(rank, world, port, q):
    """Rank 1 leaves between steps (before the timing reduction); rank 0 must get an error from
    its next collective within the process group's timeout instead of waiting for ever."""
    import datetime

    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    dist.barrier()
    if rank == 1:
        os._exit(0)  # no destroy_process_group: the peer simply goes away
    try:
        bench.max_over_ranks(1.0, world, torch.device("cpu"))
        q.put((0, "no error"))
    except Exception as e:  # gloo reports the closed connection or the timeout
        q.put((0, "error: " + type(e).__name__))


@pytest.mark.timeout(180)
def test_a_rank_that_leaves_is_detected_by_the_next_collective():
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_leaves, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    try:
        rank, msg = q.get(timeout=120)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert rank == 0 and msg.startswith("error"), msg
    assert procs[1].exitcode == 0
