"""Host-side helpers for runs over several ranks (one process per GPU).

Realisations are independent (the covariance of the multipoles comes from an
ensemble of mocks, Sec. 2), so ranks split the mock index range and exchange
nothing on the data path.  What crosses ranks is host bookkeeping: the FP64
rows of per-mock multipoles, gathered in mock order for the covariance, and
timings, combined as the slowest rank's.  The helpers take whatever process
group is initialised (NCCL with CUDA tensors on GPUs, gloo with CPU tensors)
and reduce to plain local operations when there is none or a single rank.
"""
from __future__ import annotations


def _world():
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized():
        return dist.get_rank(), dist.get_world_size()
    return 0, 1


def mock_range(n_mocks: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous share [lo, hi) of mocks 0 .. n_mocks - 1 for `rank` of
    `world`; shares differ in size by at most one and cover the range once."""
    if n_mocks < 0 or world < 1 or not 0 <= rank < world:
        raise ValueError("bad mock range request")
    return n_mocks * rank // world, n_mocks * (rank + 1) // world


def max_over_ranks(value: float, device=None) -> float:
    """The largest `value` over all ranks (the slowest rank's time)."""
    import torch
    import torch.distributed as dist

    _, world = _world()
    if world == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_rows(rows, n_mocks: int):
    """All ranks' rows [hi - lo][d] (this rank's share of `mock_range`) as one
    [n_mocks][d] tensor in mock order, on every rank, on the device of `rows`."""
    import torch
    import torch.distributed as dist

    rank, world = _world()
    lo, hi = mock_range(n_mocks, rank, world)
    if rows.dim() != 2 or rows.shape[0] != hi - lo:
        raise ValueError("rows must be [%d][d] for mocks %d .. %d" % (hi - lo, lo, hi - 1))
    if world == 1:
        return rows
    counts = [mock_range(n_mocks, r, world) for r in range(world)]
    cap = max(h - l for l, h in counts)
    d = rows.shape[1]
    pad = torch.zeros((cap, d), dtype=rows.dtype, device=rows.device)
    pad[: hi - lo] = rows
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad)
    return torch.cat([parts[r][: h - l] for r, (l, h) in enumerate(counts)], dim=0)
