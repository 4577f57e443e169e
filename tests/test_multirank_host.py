"""Host logic of the N > 1 benchmark path on CPU ranks (gloo, world size 2).

A single configuration does not shard without an exchange step, so N GPUs
run N independent replicas: the only cross-rank steps are a barrier and a
max over the ranks' times.  These tests run that logic with two CPU
processes on the gloo backend.
"""
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


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_s = [0.004, 0.007][rank]  # rank 1 is the slow replica
        t = bench.max_over_ranks(local_s, dist, "cpu")
        dist.barrier()
        q.put((rank, t, bench.whole_job_rate(100000, world, t)))
    finally:
        dist.destroy_process_group()


def test_replicas_report_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, _, _ in out] == [0, 1]
    for _, t, rate in out:
        assert t == 0.007  # both ranks see the slowest replica's time
        assert rate == pytest.approx(2 * 100000 / 0.007)  # whole-job nodes/s


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(0.25, None) == 0.25
    assert bench.whole_job_rate(10, 1, 0.5) == 20.0


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
