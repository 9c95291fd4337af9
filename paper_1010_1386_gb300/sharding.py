"""Host-side partition of independent resultants across ranks (one process
per GPU).  Resultants of different pairs share nothing, so the path shards
without any data-path collective: each rank runs its part and only the
timing is reduced.  Costs are estimates of the work per pair (e.g. images x
per-image products from the planner)."""
import heapq


def shard_by_cost(costs, world, rank):
    """Indices of the pairs rank `rank` processes: longest-processing-time
    first, each pair to the currently least-loaded rank (ties by rank)."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    heap = [(0.0, r) for r in range(world)]
    mine = []
    for i in sorted(range(len(costs)), key=lambda i: (-costs[i], i)):
        load, r = heapq.heappop(heap)
        if r == rank:
            mine.append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    return sorted(mine)


def rank_seed(base, rank):
    """Seed of rank `rank`'s own batch under weak scaling."""
    return base + 1000 * rank


def max_over_ranks(value, dist=None, device=None):
    """Maximum of a float over the ranks of the default process group (the
    value itself without one).  Works on gloo (CPU tensors) and NCCL."""
    if dist is None or not dist.is_initialized():
        return value
    import torch
    t = torch.tensor([float(value)], device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
