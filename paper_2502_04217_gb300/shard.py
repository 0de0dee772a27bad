"""Split of a batch of independent problems across ranks (one process per GPU).

The batched solve has no exchange between problems, so several GPUs share a batch
by taking disjoint subsets of it: no collective touches the data path; the ranks
only meet at a barrier and a MAX of their timings.  The split is the
longest-processing-time rule on the cost n log2 n of each problem (an FFT-bound
solve), which keeps the largest load within 4/3 of the optimum.
"""

import math


def cost(dims):
    """Work estimate of one solve on a grid of the given extents: n log2 n."""
    n = 1
    for d in dims:
        n *= int(d)
    return n * math.log2(max(n, 2))


def assign(costs, world_size):
    """Indices of the problems each rank solves: problems in order of decreasing
    cost, each to the currently lightest rank (ties: lowest rank, then lowest
    index), every index exactly once.  Returns (shares, loads)."""
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    loads = [0.0] * world_size
    shares = [[] for _ in range(world_size)]
    for i in order:
        r = min(range(world_size), key=lambda k: (loads[k], k))
        loads[r] += costs[i]
        shares[r].append(i)
    return [sorted(s) for s in shares], loads


def rank_share(dims_list, world_size, rank):
    """The sorted problem indices of one rank for a batch given by its grid extents."""
    shares, _ = assign([cost(d) for d in dims_list], world_size)
    return shares[rank]


def max_over_ranks(value, dist=None, device=None):
    """MAX of a float over the ranks of the default process group (the value
    itself without one)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
