"""Multi-rank host logic on CPU: two gloo ranks split a mock range, gather
their FP64 rows in mock order and take the slowest rank's time.  No GPU."""
import os
import socket

import numpy as np
import pytest

from paper_1708_05303_gb300.dist import mock_range


@pytest.mark.parametrize("n,world", [(0, 2), (1, 2), (7, 2), (512, 3), (5, 8)])
def test_mock_range_partitions(n, world):
    seen = []
    sizes = []
    for r in range(world):
        lo, hi = mock_range(n, r, world)
        seen.extend(range(lo, hi))
        sizes.append(hi - lo)
    assert seen == list(range(n))
    assert max(sizes) - min(sizes) <= 1


def test_mock_range_rejects_bad_requests():
    for args in [(-1, 0, 1), (4, 2, 2), (4, 0, 0)]:
        with pytest.raises(ValueError):
            mock_range(*args)


def _row(m, d):
    return np.array([m + 0.25 * j + 1e-3 * m * j for j in range(d)], dtype=np.float64)


def _rank_main(rank, world, port, n, d, q):
    import torch
    import torch.distributed as dist

    from paper_1708_05303_gb300.dist import gather_rows, max_over_ranks

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        lo, hi = mock_range(n, rank, world)
        rows = torch.from_numpy(np.stack([_row(m, d) for m in range(lo, hi)]) if hi > lo
                                else np.zeros((0, d)))
        full = gather_rows(rows, n)
        slow = max_over_ranks(1.5 + rank)   # rank r "took" 1.5 + r ms
        q.put((rank, full.numpy().tolist(), slow))
    finally:
        dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


@pytest.mark.parametrize("n", [7, 2])
def test_gather_rows_and_max_over_two_gloo_ranks(n):
    import torch.multiprocessing as mp

    world, d = 2, 5
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, n, d, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(world):
        rank, full, slow = q.get(timeout=120)
        out[rank] = (np.array(full), slow)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want = np.stack([_row(m, d) for m in range(n)])
    for rank in range(world):
        full, slow = out[rank]
        assert np.array_equal(full, want)      # every rank holds all rows, in mock order
        assert slow == 1.5 + (world - 1)       # the slowest rank's time
