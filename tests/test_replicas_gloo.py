"""The N > 1 benchmark path runs independent replicas (the operator apply has no data-path
collective on one GPU per rank): the only exchange is the max over ranks of the timed region.
Checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seconds = 1.0 + 0.5 * rank                       # the second rank is slower
    t = bench.max_over_ranks(seconds, dist, "cpu")
    rate = bench.whole_job_rate(6_714_692, 10, world, t)
    dist.barrier()
    out[rank] = (t, rate)
    dist.destroy_process_group()


def test_two_gloo_ranks_time_the_slowest_replica():
    import torch.multiprocessing as mp
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 1.5
    assert res[0][1] == pytest.approx(6_714_692 * 10 * 2 / 1.5 / 1e9)
