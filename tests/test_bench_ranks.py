"""The multi-rank path of bench.py on the CPU: two gloo ranks (127.0.0.1)
run the same rank helpers the GPU launch uses (barrier on both sides of the
timed region, time = maximum over ranks, one independent cluster per rank,
whole-job rate over all ranks), and the reference arm leaves the work to
rank 0."""
import contextlib
import io
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as tdist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r = bench.Ranks(rank, world, "cpu")
        r.barrier()
        local_ms = 10.0 + 5.0 * rank  # rank 1 is the slower one
        ms = r.max(local_ms)
        r.barrier()
        value = bench.whole_job_rate(1000, 4, world, ms)
        # the reference arm: only rank 0 works and prints
        out = io.StringIO()
        args = type("A", (), {})()
        if rank != 0:
            with contextlib.redirect_stdout(out):
                bench.run_reference(args, rank, world)
        q.put((rank, ms, value, bench.replica_seed(7, rank), out.getvalue()))
    finally:
        tdist.destroy_process_group()


def test_two_gloo_ranks_time_the_slowest_and_aggregate():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
    assert all(p.exitcode == 0 for p in ps)
    res = sorted(q.get(timeout=5) for _ in range(world))
    assert [x[1] for x in res] == [15.0, 15.0]  # both see the slower rank's time
    assert res[0][2] == res[1][2] == 1000 * 4 * 2 / 0.015
    assert res[0][3] != res[1][3]  # independent clusters
    assert res[1][4] == ""  # rank 1 of the reference arm prints nothing


def test_single_rank_helpers():
    r = bench.Ranks(0, 1, "cpu")
    r.barrier()
    assert r.max(3.5) == 3.5
    assert bench.whole_job_rate(10, 2, 1, 1000.0) == 20.0
    assert bench.replica_seed(1, 0) == 1
