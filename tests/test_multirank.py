"""The multi-rank logic of bench.py on CPU: two gloo ranks reduce their timings to the
slowest rank's, and the whole-job rate counts every rank's cells (weak scaling)."""
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
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took (1 + r) s for the steps and 10 - r ms per launch
        got = bench.max_over_ranks([1.0 + rank, 10.0 - rank], world, "cpu")
        out[rank] = got + [bench.job_rate(world, 1000, 4, got[0])]
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_timing():
    world, port = 2, _free_port()
    with mp.get_context("spawn").Manager() as m:  # no fork of this multi-threaded process
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        assert res[r][:2] == [2.0, 10.0]
        assert res[r][2] == pytest.approx(2 * 1000 * 4 / 2.0)


def test_single_rank_is_the_identity():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    assert bench.max_over_ranks([3.0, 4.0], 1, "cpu") == [3.0, 4.0]
    assert bench.job_rate(1, 10, 2, 4.0) == 5.0
