"""World-size-2 gloo tests (CPU) of the multi-rank host path: the cost-based
partition is disjoint and complete and balanced, and the max-over-ranks
reduction that the benchmark uses agrees on every rank."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as tmp

from paper_1010_1386_gb300 import sharding


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, costs, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = sharding.shard_by_cost(costs, world, rank)
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    m = sharding.max_over_ranks(10.0 + rank, dist)
    load = sum(costs[i] for i in mine)
    loads = [None] * world
    dist.all_gather_object(loads, load)
    out[rank] = (gathered, m, loads)
    dist.barrier()
    dist.destroy_process_group()


def test_partition_and_reduction_on_two_gloo_ranks():
    costs = [((i * 7919) % 97) + 1 for i in range(40)]
    mgr = tmp.Manager()
    out = mgr.dict()
    tmp.spawn(_worker, args=(2, _free_port(), costs, out), nprocs=2, join=True)
    g0, m0, loads = out[0]
    g1, m1, _ = out[1]
    assert g0 == g1
    a, b = set(g0[0]), set(g0[1])
    assert not (a & b) and a | b == set(range(40))
    assert m0 == m1 == 11.0
    assert abs(loads[0] - loads[1]) <= max(costs)


def test_single_rank_is_everything():
    assert sharding.shard_by_cost([3, 1, 2], 1, 0) == [0, 1, 2]
    with pytest.raises(ValueError):
        sharding.shard_by_cost([1], 2, 2)
    assert sharding.max_over_ranks(4.5) == 4.5
    assert sharding.rank_seed(2, 0) == 2 and sharding.rank_seed(2, 3) == 3002
