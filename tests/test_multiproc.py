"""bench.py's multi-rank path on CPU: two gloo ranks, each timing its own replica; the job
time is the maximum over ranks and the throughput counts every rank's views."""
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


def _rank(rank: int, world: int, port: int, q) -> None:
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    mine = [10.0 + rank, 3.0 - rank, 7.0]
    got = bench.reduce_max(mine, device="cpu")
    dist.barrier()
    q.put((rank, got, bench.throughput(50, 20, world, got[0])))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_and_count_all_views():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, tput in out:
        assert got == [11.0, 3.0, 7.0]
        assert tput == pytest.approx(2 * 50 * 20 / 0.011)


def test_single_process_is_identity():
    import bench
    assert bench.reduce_max([1.5, 2.5]) == [1.5, 2.5]
    assert bench.throughput(50, 10, 1, 1000.0) == pytest.approx(500.0)
