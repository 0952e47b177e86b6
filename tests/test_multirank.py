"""The multi-rank host logic of bench.py (one independent beam per rank, a
barrier around the timed region, the maximum time over ranks, rank 0 alone
reporting) on two gloo ranks on the CPU."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.barrier(world)
    t = bench.max_over_ranks(10.0 + 5.0 * rank, world, torch.device("cpu"))
    # the reference arm: rank 0 alone runs and prints, the others return at once
    buf = io.StringIO()

    class A:
        steps, warmup, gpus = 0, 0, world
    if rank != 0:
        with redirect_stdout(buf):
            bench.run_reference(A)
    bench.barrier(world)
    q.put((rank, t, buf.getvalue()))
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_rank0_reporting():
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
    assert [o[1] for o in out] == [15.0, 15.0]          # both ranks see the slowest time
    assert out[1][2] == ""                              # a non-zero rank prints nothing
