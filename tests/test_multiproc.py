"""The N > 1 path of bench.py as independent replicas: two gloo ranks on CPU (no GPU), the
max-over-ranks timing, the whole-job throughput and distinct replica seeds."""
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


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, local = bench.dist_env()
    ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
    worst = bench.reduce_max(ms, dist, device="cpu")
    value = bench.job_value(1000, w, worst * 1e-3)
    out[rank] = (w, r, local, worst, value, bench.replica_seed(3, r))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_sum_the_units():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    for rank, (w, r, local, worst, value, seed) in res.items():
        assert (w, r, local) == (2, rank, rank)
        assert worst == 15.0                      # max over ranks
        assert value == pytest.approx(2000 / 0.015)  # both ranks' units over the slowest time
    assert res[0][5] != res[1][5]                 # independent replicas
