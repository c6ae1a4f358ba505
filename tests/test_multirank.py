"""The multi-GPU form of the bench (one replica of the relaxation per rank,
no data-path collective): its host logic on two gloo ranks on the CPU.  Each
rank reports its own timed-region length; every rank must see the slowest
one, and the whole-job throughput counts every rank's relaxations over that
time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.env_rank()
        assert (r, w, local) == (rank, world, rank)
        ms = 100.0 + 50.0 * rank                 # rank 1 is the slow one
        ms_max = bench.max_over_ranks(ms, world)
        out[rank] = (ms_max, bench.throughput(5, world, ms_max))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    port = _free_port()
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]
    ms_max, value = res[0]
    assert ms_max == 150.0
    assert value == pytest.approx(2 * 5 / 0.150)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.throughput(3, 1, 500.0) == pytest.approx(6.0)
