"""Host logic of the multi-rank bench, run as two gloo ranks on the CPU.

Under torchrun every rank predicts its own human with no data-path
collective; the job's value is all ranks' particle-steps over the slowest
rank's time, and the reference arm prints from rank 0 only.
"""
import contextlib
import io
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as tdist

    import bench

    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        slow = bench.max_over_ranks(times[rank], world, tdist, "cpu")
        value = bench.job_throughput(world, 1000, slow)
        ids = [None] * world
        tdist.all_gather_object(ids, bench.rank_human_id(1, rank))
        tdist.barrier()
        q.put((rank, slow, value, ids))
    finally:
        tdist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_shard_by_human():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    times = [0.5, 0.8]
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slow, value, ids in out:
        assert slow == pytest.approx(0.8)
        assert value == pytest.approx(2 * 1000 / 0.8)  # both ranks' units over the slowest time
        assert len(set(ids)) == 2                      # each rank has its own human


def test_rank_humans_draw_independent_streams(orc):
    import bench

    a = orc.philox4x64([0, 0, 2, 0], [7, bench.rank_human_id(1, 0)])
    b = orc.philox4x64([0, 0, 2, 0], [7, bench.rank_human_id(1, 1)])
    assert not np.array_equal(a, b)


def test_reference_arm_prints_on_rank_zero_only(monkeypatch):
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        steps, warmup, cpu_sample = 1, 0, 1000

    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(A())
    assert buf.getvalue() == ""


def test_single_rank_needs_no_process_group():
    import bench

    assert bench.max_over_ranks(1.25, 1) == 1.25
    assert bench.job_throughput(1, 15_000_000, 0.5) == 30_000_000
