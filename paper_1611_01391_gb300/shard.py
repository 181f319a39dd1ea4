"""Independent units over several GPUs: which rank solves which unit, and
the final gather of the results to rank 0.

One C-A solve is a chain of data-dependent decisions, so it stays on one
GPU; what spreads over GPUs are independent units: the far-field blocks of
one batched job (Section 9) and the requests of the served form.  Each rank
(one process per GPU) solves its own share with the library and nothing is
exchanged until the end, when rank 0 gathers (I, J, U) of every unit.  This
module is host logic only (plain Python plus torch.distributed for the
gather); the solves themselves run in the library's kernels.
"""
from __future__ import annotations

import heapq


def block_costs(blocks, l):
    """Work estimate of each block of a batched job: (m_b + n_b) l_b entries
    per sweep (the two strips of a C-A sweep), with l_b the block's cross
    size (a scalar for all blocks, or one per block)."""
    out = []
    for b, blk in enumerate(blocks):
        lb = l if isinstance(l, (int, float)) else l[b]
        out.append(float((int(blk[1]) + int(blk[3])) * lb))
    return out


def lpt_partition(costs, world):
    """Longest Processing Time first (Graham 1969): units by decreasing cost
    (ties: the smaller index first), each to the rank with the least work
    so far (ties: the lower rank).  Every unit goes to exactly one rank;
    the largest load is at most (4/3 - 1/(3 world)) of the best possible.
    Returns one ascending index list per rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0.0, r) for r in range(world)]
    parts = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    return [sorted(p) for p in parts]


def route_requests(costs, world, start=0):
    """Served requests in arrival order to ranks: each to the rank with the
    shortest queue (least estimated work assigned so far); ties go round
    robin, to the first tied rank at or after the one following the previous
    choice (`start` for the first request).  Returns the rank of each
    request."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0.0] * world
    nxt = start % world
    out = []
    for c in costs:
        best = min(load)
        r = next((nxt + k) % world for k in range(world) if load[(nxt + k) % world] == best)
        out.append(r)
        load[r] += c
        nxt = (r + 1) % world
    return out


def gather_to_root(local, world, rank):
    """Merge the ranks' {unit index: result} dictionaries on rank 0 (the
    only collective, after every solve has finished).  Returns the merged
    dictionary on rank 0 and None elsewhere; a unit reported by two ranks
    is an error."""
    if world <= 1:
        return dict(local)
    import torch.distributed as dist
    parts = [None] * world if rank == 0 else None
    dist.gather_object(dict(local), parts, dst=0)
    if rank != 0:
        return None
    merged = {}
    for p in parts:
        for k, v in p.items():
            if k in merged:
                raise RuntimeError(f"unit {k} solved by two ranks")
            merged[k] = v
    return merged
