"""Multi-process path of bench.py on the CPU: two gloo ranks, the way
torchrun runs one replica per GPU.  The whole-job rate is the units of all
ranks over the slowest rank's time."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        # rank r processed 100 * (r + 1) units in 1 + r seconds
        rate = bench.replica_throughput(100.0 * (rank + 1), 1.0 + rank)
        slowest = bench._reduce(1.0 + rank, "max")
        total = bench._reduce(100.0 * (rank + 1), "sum")
        out.put((rank, rate, slowest, total, bench._dist()))
    finally:
        dist.destroy_process_group()


def test_replica_reductions_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, rate, slowest, total, d in res:
        assert slowest == 2.0          # the slowest rank's time
        assert total == 300.0          # the units of all ranks
        assert rate == pytest.approx(150.0)  # 300 units / 2 s, the same on every rank
        assert d == (world, rank, rank)


def test_replica_throughput_one_process():
    sys.path.insert(0, ROOT)
    import bench
    assert not dist.is_initialized()
    assert bench.replica_throughput(287048 * 100, 0.4) == pytest.approx(287048 * 250)
