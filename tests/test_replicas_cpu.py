"""The multi-GPU path is replicas only (one elimination per rank, no data-path
collective): the benchmark's only cross-rank steps are the barrier and the
max-over-ranks reduction of the step time. Those run here on two gloo ranks."""
from __future__ import annotations

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    dist.barrier()
    step_ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
    mx = bench.max_over_ranks(step_ms, world)
    out.put((rank, mx, bench.job_seconds_per_matrix(mx, world)))
    dist.destroy_process_group()


def test_max_over_ranks_and_job_value_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every rank sees the slowest rank's time; the job completes two matrices per step
    assert [r[1] for r in res] == [15.0, 15.0]
    assert res[0][2] == pytest.approx(15.0 / 1e3 / 2)


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_seconds_per_matrix(20.0, 1) == pytest.approx(0.02)
