"""The N > 1 host path of bench.py on CPU ranks (gloo, world size 2):
barrier, MAX of the elapsed time over ranks, whole-job throughput, and the
reference arm's rank handling (rank 0 alone runs; the others exit without
work or output)."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout
from types import SimpleNamespace

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    dist.barrier()
    mine = [3.5, 5.25][rank]
    worst = bench.max_over_ranks(mine, torch, dist, "cpu")
    value = bench.job_throughput(world, 1000, 10, worst)
    out = io.StringIO()
    with redirect_stdout(out):
        r = bench.run_reference_arm(SimpleNamespace(steps=1, warmup=0), rank, world) if rank == 1 else None
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, worst, value, r, out.getvalue()))


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, worst, value, r, printed in res:
        assert worst == 5.25
        assert value == pytest.approx(2 * 1000 * 10 / 5.25e-3)
    # the reference arm's rank 1 returns at once and prints nothing
    assert res[1][3] is None and res[1][4] == ""
