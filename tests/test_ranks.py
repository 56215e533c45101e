"""Multi-rank host logic on CPU (gloo, world size 2): the cell shards (equal counts and equal
predicted cost), the max-over-ranks timing and the sum of the per-rank ln A gradients (the
adjoint's exchange step)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2105_12070_gb300 import ranks  # noqa: E402


def test_shard_range_covers_every_cell_once():
    for n in (0, 1, 7, 65536, 65537):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                a, b = ranks.shard_range(n, r, world)
                assert 0 <= a <= b <= n
                seen.extend(range(a, b))
            assert seen == list(range(n))
            sizes = [ranks.shard_range(n, r, world)[1] - ranks.shard_range(n, r, world)[0] for r in range(world)]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        ranks.shard_range(10, 2, 2)


def test_shard_by_cost_balances_contiguous_blocks():
    rng = np.random.default_rng(3)
    # a shear-layer-like cost profile: cheap pure streams, an expensive mixing band
    n = 4096
    cost = np.ones(n)
    cost[1800:2300] = rng.uniform(20.0, 200.0, size=500)
    for world in (1, 2, 3, 8):
        blocks = [ranks.shard_by_cost(cost, r, world) for r in range(world)]
        assert blocks[0][0] == 0 and blocks[-1][1] == n
        assert all(blocks[r][1] == blocks[r + 1][0] for r in range(world - 1))
        loads = np.array([cost[a:b].sum() for a, b in blocks])
        assert loads.sum() == cost.sum()
        assert loads.max() <= cost.sum() / world + cost.max()
        if world > 1:
            equal = [cost[a:b].sum() for a, b in (ranks.shard_range(n, r, world) for r in range(world))]
            assert loads.max() < max(equal)  # better than equal cell counts on this profile
    # degenerate inputs
    assert ranks.shard_by_cost(np.zeros(10), 1, 2) == ranks.shard_range(10, 1, 2)
    assert [ranks.shard_by_cost([5.0], r, 3) for r in range(3)] == [(0, 1), (1, 1), (1, 1)]
    assert ranks.shard_by_cost([], 0, 2) == (0, 0)
    with pytest.raises(ValueError):
        ranks.shard_by_cost([1.0, -1.0], 0, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # per-cell ln A gradients of 10 cells and 3 reactions, split over the ranks
        rng = np.random.default_rng(0)
        g_cells = rng.normal(size=(10, 3))
        a, b = ranks.shard_range(10, rank, world)
        g = torch.from_numpy(g_cells[a:b].sum(axis=0).copy())
        ranks.sum_lnA_grad(g)
        times = ranks.max_over_ranks([1.0 + rank, 5.0 - rank])
        # each rank takes its cost-balanced block; gathered, the blocks tile the cells once
        cost = rng.uniform(1.0, 50.0, size=101)
        mine = torch.tensor(ranks.shard_by_cost(cost, rank, world), dtype=torch.int64)
        allb = [torch.zeros(2, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(allb, mine)
        q.put((rank, g.numpy().tolist(), times, g_cells.sum(axis=0).tolist(), [b.tolist() for b in allb]))
    finally:
        dist.destroy_process_group()


def test_gloo_two_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, g, times, want, blocks in out:
        np.testing.assert_allclose(g, want, rtol=1e-14, atol=1e-14)
        assert times == [2.0, 5.0]
        assert blocks[0][0] == 0 and blocks[0][1] == blocks[1][0] and blocks[1][1] == 101


def test_single_process_is_identity():
    g = torch.arange(3, dtype=torch.float64)
    assert ranks.sum_lnA_grad(g) is g
    assert ranks.max_over_ranks([1.5, 2.5]) == [1.5, 2.5]
