"""bench.py's multi-process path on the CPU: under torchrun every rank solves its own replica (no
collective on the data path) and the job's time is the slowest rank's; the reference arm runs on
rank 0 only.  Two gloo processes stand in for two GPUs."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, ms, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist = bench.init_replicas()
    out = bench.slowest_rank_ms(ms, dist)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, out))


def test_slowest_rank_over_two_gloo_processes():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    times = [12.5, 31.25]
    procs = [ctx.Process(target=_rank, args=(r, 2, port, times[r], q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == {0: max(times), 1: max(times)}


def test_one_process_has_no_group():
    sys.path.insert(0, ROOT)
    import bench
    old = os.environ.pop("WORLD_SIZE", None)
    try:
        assert bench.init_replicas() is None
        assert bench.slowest_rank_ms(7.0, None) == 7.0
    finally:
        if old is not None:
            os.environ["WORLD_SIZE"] = old


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
