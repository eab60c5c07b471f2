"""Multi-rank logic of bench.py on CPU ranks (gloo, world size 2): the timed value is
the slowest rank's, the job value counts every rank's cell updates, and the
reference arm prints from rank 0 only."""
import io
import multiprocessing as mp
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

from conftest import ROOT


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.reduce_max(100.0 + 7.0 * rank, dist, "cpu")
    value = bench.job_value(world, 1000, 10, ms)
    args = type("A", (), dict(n=32, steps=1, warmup=0, gpus=world))()
    buf = io.StringIO()
    if rank == 1:  # a non-zero rank of the reference arm exits without work or output
        with redirect_stdout(buf):
            bench.run_reference(args)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ms, value, buf.getvalue()))


def test_two_gloo_ranks_aggregate_like_the_benchmark():
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value, out in res:
        assert ms == 107.0  # max over ranks
        assert value == pytest.approx(2 * 1000 * 10 / 0.107 / 1e6)
    assert res[1][3] == ""
