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


# ---------------------------------------------------------------------------
# Independent units over ranks: LPT split of one block list, shortest-queue
# routing of requests, gather of the results to rank 0 (host logic, CPU)
# ---------------------------------------------------------------------------

def test_lpt_partition_is_exact_and_within_grahams_bound():
    import itertools
    import random
    from paper_1611_01391_gb300.shard import lpt_partition
    rnd = random.Random(3)
    for world in (2, 3):
        for _ in range(20):
            costs = [rnd.randint(1, 50) for _ in range(8)]
            parts = lpt_partition(costs, world)
            assert sorted(i for p in parts for i in p) == list(range(8))   # each unit exactly once
            span = max(sum(costs[i] for i in p) for p in parts)
            best = min(max(sum(c for c, r in zip(costs, a) if r == q) for q in range(world))
                       for a in itertools.product(range(world), repeat=8))
            assert span <= (4 / 3 - 1 / (3 * world)) * best + 1e-9, (costs, span, best)


def test_lpt_partition_ties_and_costs():
    from paper_1611_01391_gb300.shard import block_costs, lpt_partition
    assert lpt_partition([1, 1, 1, 1], 2) == [[0, 2], [1, 3]]
    blocks = [[0, 100, 0, 50, ], [0, 10, 0, 10], [0, 300, 0, 200]]
    assert block_costs(blocks, 12) == [1800.0, 240.0, 6000.0]
    assert block_costs(blocks, [12, 24, 6]) == [1800.0, 480.0, 3000.0]
    assert lpt_partition(block_costs(blocks, 12), 2) == [[2], [0, 1]]


def test_route_requests_shortest_queue_round_robin():
    from paper_1611_01391_gb300.shard import route_requests
    assert route_requests([1, 1, 1, 1, 1], 2) == [0, 1, 0, 1, 0]
    assert route_requests([10, 1, 1, 1], 2) == [0, 1, 1, 1]
    assert route_requests([1, 1, 1], 3, start=2) == [2, 0, 1]


def _solve_share(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    if world > 1:
        dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import numpy as np
        import oracle as O
        import workloads as W
        from paper_1611_01391_gb300.shard import block_costs, gather_to_root, lpt_partition
        from tests._parity import SubSource
        pts, blocks = W.octree_block_pairs(11, npoints=1 << 12, leaf=64, n_pairs=10)
        jc, sr, sc = W.block_candidates(12, blocks, 24, 8)
        share = lpt_partition(block_costs(blocks, 12), world)[rank]
        src = O.InvDist(pts, pts, "fp32")
        local = {}
        for b in share:
            r0, m, c0, n = (int(v) for v in blocks[b])
            I, J, U, k, s, l, sw = O.cross_approximation_adaptive(SubSource(src, r0, m, c0, n), jc[b], 12, 24, 16,
                                                                  2, 1e-6, sample_rows=sr[b], sample_cols=sc[b])
            local[b] = (list(I), list(J), np.asarray(U).tolist())
        merged = gather_to_root(local, world, rank)
        if rank == 0:
            out["merged"] = merged
            out["n_blocks"] = len(blocks)
        out[f"share{rank}"] = share
    finally:
        if world > 1:
            dist.destroy_process_group()


def test_two_ranks_solve_every_block_once_and_match_one_rank():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_solve_share, args=(world, port, out), nprocs=world, join=True)
        two = dict(out)
        one = {}
        _solve_share(0, 1, port, one)
    assert set(two["share0"]).isdisjoint(two["share1"])
    assert sorted(two["merged"]) == list(range(two["n_blocks"])) == sorted(one["merged"])
    for b in range(two["n_blocks"]):
        assert two["merged"][b] == one["merged"][b]
