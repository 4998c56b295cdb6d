"""The multi-rank host logic of the benchmark on CPU (gloo, world size 2).

One process per GPU, each running the whole batch (weak scaling, no
collective on the data path): the step time is the maximum over ranks, the
value counts every rank's matrices, and the reference arm runs on rank 0 only.
"""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch
    import bench
    w, r, _ = bench.ranks_setup("gloo")
    bench.rank_barrier(w)
    local_ms = 10.0 * (r + 1)  # rank 1 is the slower one
    ms = bench.rank_max(local_ms, w, torch.device("cpu"))
    q.put((r, w, ms, bench.whole_job_value(w, 4096, ms)))
    bench.rank_barrier(w)
    torch.distributed.destroy_process_group()


def test_two_ranks_max_time_and_whole_job_value():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for r, (rank, w, ms, value) in enumerate(out):
        assert rank == r and w == 2
        assert ms == 20.0                      # the slowest rank's time
        assert value == 2 * 4096 / 0.020       # both ranks' matrices


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.rank_max(3.5, 1, None) == 3.5
    assert bench.whole_job_value(1, 4096, 200.0) == 4096 / 0.2


def test_reference_arm_other_ranks_exit_without_work():
    """Under torchrun only rank 0 times the oracle; the others exit 0 at once."""
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
