"""The bench's multi-rank path on CPU (gloo, world size 2).

The solver does not shard (every round of a phase needs a global minimum per
column), so `bench.py --gpus N` runs N independent replicas: each rank times
its own solves between barriers, the job time is the maximum over ranks, and
the reported per-solve time divides it by all solves of all ranks.  The
reference arm runs on rank 0 only.
"""
import importlib.util
import io
import os
import socket
import contextlib

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = load_bench()
        dist.barrier()
        # rank r "took" 10 + 5 r ms for its 4 steps
        total = b.max_over_ranks(10.0 + 5.0 * rank, dist, torch.device("cpu"))
        per_step, job = b.job_time(total, 4, world)
        # the reference arm: only rank 0 prints its line
        buf = io.StringIO()

        class A:
            n, seed, eps, warmup, steps, gpus = 64, 0, 0.1, 0, 1, world
        with contextlib.redirect_stdout(buf):
            b.run_reference(A, world, rank)
        q.put((rank, total, per_step, job, buf.getvalue().strip()))
    finally:
        dist.destroy_process_group()


def test_replicas_take_the_slowest_rank():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for rank, total, per_step, job, line in out:
        assert total == 15.0                 # the slower rank's time, on every rank
        assert per_step == 15.0 / 4
        assert job == 15.0 / 4 / world       # world * 4 solves in 15 ms
        if rank == 0:
            assert '"impl": "reference"' in line
        else:
            assert line == ""                # other ranks do no work and print nothing


def test_single_rank_is_unchanged():
    b = load_bench()
    assert b.max_over_ranks(7.5, None, None) == 7.5
    assert b.job_time(30.0, 3, 1) == (10.0, 10.0)
