"""Multi-GPU host logic on CPU: the split of independent structures across ranks
and the max-over-ranks timing, with two gloo ranks (no GPU)."""
import os
import socket

import numpy as np
import pytest

from paper_2607_17978_b300 import shard


def test_partition_covers_every_index_once_and_balances():
    rng = np.random.default_rng(0)
    costs = np.exp(rng.uniform(np.log(64), np.log(4096), size=512))
    for n in (1, 2, 3, 4, 8):
        parts = shard.partition(costs, n)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        loads = [costs[p].sum() for p in parts]
        assert max(loads) <= costs.sum() / n + costs.max() + 1e-9
        assert parts == shard.partition(costs, n)  # deterministic


def test_partition_meets_grahams_bound_against_brute_force():
    """Largest-first greedy scheduling on m parts has makespan <= (4/3 - 1/(3m)) of the optimum
    (Graham 1969); the optimum here is found by trying every assignment of small batches."""
    import itertools
    rng = np.random.default_rng(2)
    for trial in range(60):
        m = int(rng.integers(2, 4))
        costs = [float(c) for c in rng.integers(1, 50, size=int(rng.integers(m + 1, 9)))]
        greedy = max(sum(costs[i] for i in p) for p in shard.partition(costs, m))
        best = min(max(sum(c for c, a in zip(costs, assign) if a == k) for k in range(m))
                   for assign in itertools.product(range(m), repeat=len(costs)))
        assert best <= greedy <= (4.0 / 3.0 - 1.0 / (3 * m)) * best + 1e-9, (costs, m)


def test_partition_edge_cases():
    assert shard.partition([], 3) == [[], [], []]
    assert shard.partition([5.0], 2) == [[0], []]
    assert shard.partition([1.0, 1.0, 1.0, 1.0], 2) == [[0, 2], [1, 3]]
    with pytest.raises(ValueError):
        shard.partition([1.0], 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, costs, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = shard.rank_share(costs, rank, world)
        shares = [None] * world
        dist.all_gather_object(shares, mine)
        t_max = shard.max_over_ranks(1.0 + rank)
        n_sum = shard.sum_over_ranks(float(len(mine)))
        out.put((rank, shares, t_max, n_sum))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_split_the_batch_and_agree_on_the_step_time():
    import torch.multiprocessing as mp
    costs = [float(n) for n in np.random.default_rng(1).integers(64, 4096, size=37)]
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, costs, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, shares, t_max, n_sum in res:
        flat = sorted(i for s in shares for i in s)
        assert flat == list(range(len(costs)))      # every structure on exactly one rank
        assert shares == shard.partition(costs, world)
        assert t_max == 2.0                          # the slowest rank sets the step time
        assert n_sum == len(costs)
