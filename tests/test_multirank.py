"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2): each
rank solves its own units (distinct seeds), and the timed region is the
maximum over ranks.  No GPU and no collective on the data path."""
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


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        got = bench.max_over_ranks(10.0 * (rank + 1), world, "cpu")
        inp = bench.make_inputs(bench.WORKLOADS["dense256"], rank)
        out[rank] = (got, inp["J0"].tolist())
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_distinct_units():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 20.0          # every rank sees the slowest rank's time
    assert res[0][1] != res[1][1]                  # each rank draws its own units


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
