"""Multi-rank host logic on CPU (gloo, world size 2): the cell shards, the max-over-ranks timing
and the sum of the per-rank ln A gradients (the adjoint's exchange step)."""
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
        q.put((rank, g.numpy().tolist(), times, g_cells.sum(axis=0).tolist()))
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
    for rank, g, times, want in out:
        np.testing.assert_allclose(g, want, rtol=1e-14, atol=1e-14)
        assert times == [2.0, 5.0]


def test_single_process_is_identity():
    g = torch.arange(3, dtype=torch.float64)
    assert ranks.sum_lnA_grad(g) is g
    assert ranks.max_over_ranks([1.5, 2.5]) == [1.5, 2.5]
