"""The multi-rank logic of the bench on CPU: two gloo ranks (one per GPU in a
multi-GPU run, replicas with no data-path collective) must agree on the
job's time — the slowest rank's — and on the whole-job rate."""
from __future__ import annotations

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 10.0 + 5.0 * rank                    # the ranks take different times
    t = bench.max_over_ranks(ms, dist, "cpu")
    rate = bench.whole_job_rate(world, 1000, 4, t)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, t, rate))


def test_two_gloo_ranks_agree_on_time_and_rate():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, t, rate in res:
        assert t == 15.0                       # the slowest rank's time
        assert rate == pytest.approx(2 * 1000 * 4 / 0.015)


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.whole_job_rate(1, 10, 2, 1.0) == pytest.approx(20_000.0)
