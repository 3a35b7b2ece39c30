"""The multi-process path of bench.py on CPU: two gloo ranks.

On N GPUs every rank runs its own lattice (replicas, no collective on the
data path). The only cross-rank steps are the maximum of the timed
durations and rank 0 alone printing the line; the reference arm runs on
rank 0 only. These run here as two spawned processes on the gloo backend.
"""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # each rank's own timings; the job takes every value's slowest rank
        mine = [1.0 + rank, 5.0 - rank, 2.5]
        got = bench.max_over_ranks(mine, "cpu")
        ws, r, _ = bench.dist_setup()
        rate = bench.job_rate(ws, 1000, got[0])
        # the reference arm: rank 0 alone runs and prints, the others exit 0
        out = io.StringIO()
        if rank != 0:
            class A:
                steps, warmup = 1, 3
            with redirect_stdout(out):
                rc = bench.run_reference(A())
        else:
            rc = 0
        dist.barrier()
        q.put((rank, got, ws, r, rate, rc, out.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank_and_only_rank0_reports():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, ws, r, rate, rc, printed in res:
        assert got == [2.0, 5.0, 2.5]
        assert ws == 2 and r == rank
        assert rate == pytest.approx(2 * 1000 / 2.0)
        assert rc == 0
        if rank == 1:
            assert printed == ""  # the reference arm prints on rank 0 only
