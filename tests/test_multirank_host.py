"""The benchmark's multi-rank logic on CPU: two gloo ranks, each a replica
with its own time; every rank sees the slowest time and the whole-job value
counts both ranks' work."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        r, w, lr = bench.dist_env()
        assert (r, w, lr) == (rank, world, rank)
        ms = 10.0 + 5.0 * rank  # rank 1 is the slow replica
        got = bench.max_over_ranks(ms, device="cpu")
        out[rank] = (got, bench.whole_job_gbs(1e9, 2, w, got))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world, port = 2, _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]
    ms, gbs = res[0]
    assert ms == 15.0
    assert gbs == pytest.approx(1e9 * 2 * 2 / 15e-3 / 1e9)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(7.5, device="cpu") == 7.5
