"""The multi-rank path of bench.py on CPU: two gloo ranks (127.0.0.1), each
with its own timing, must agree on the slowest rank's time, and the
whole-job value counts the units of every rank (weak scaling)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 100.0 + 37.5 * rank                    # rank 1 is the slow one
    ms = bench.max_over_ranks(local_ms, dist, "cpu")
    e2e = bench.max_over_ranks(2.0 - rank, dist, "cpu")
    dist.barrier()
    out[rank] = (ms, e2e, bench.whole_job_mlups(world, 1_000_000, 10, ms / 1e3),
                 bench.rank_seed(20241111, rank))
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 137.5            # max over ranks, on every rank
    assert res[0][1] == res[1][1] == 2.0
    assert res[0][2] == pytest.approx(2 * 1_000_000 * 10 / 0.1375 / 1e6)
    assert res[0][3] != res[1][3]                     # independent noise per rank


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.whole_job_mlups(1, 65536 * 24, 100, 0.01) == pytest.approx(15728.64)
