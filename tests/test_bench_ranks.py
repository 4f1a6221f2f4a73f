"""The benchmark's replica logic for N > 1 ranks, on CPU with gloo and two
processes: barriers around the timed region, the slowest rank's time, and
the whole-job value (units of all ranks over that time)."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    r, w = bench.rank_world()
    bench.init_ranks(w, backend="gloo")
    bench.barrier(w)
    mine = 10.0 + 5.0 * r                  # each rank's timed total (ms)
    worst = bench.max_over_ranks(mine, w, device="cpu")
    bench.barrier(w)
    value = bench.whole_job_value(1000, w, worst)
    import torch.distributed as dist
    dist.destroy_process_group()
    q.put((r, w, worst, value))


@pytest.mark.parametrize("world", [2])
def test_two_gloo_ranks_take_the_slowest_time(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    slowest = 10.0 + 5.0 * (world - 1)
    for r, (rank, w, worst, value) in enumerate(got):
        assert rank == r and w == world and worst == slowest
        assert value == pytest.approx(1000 * world / (slowest / 1000.0))


def test_one_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    bench.init_ranks(1)
    bench.barrier(1)
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_value(2_000_000, 1, 31.4) == pytest.approx(2_000_000 / 0.0314)
