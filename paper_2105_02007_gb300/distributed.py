"""Multi-rank MLMC estimate (host side, torch.distributed).

Samples are independent, so the (level, sample index) ranges of one
allocation are split over the ranks: rank r of W solves the contiguous
samples shard(N_l, r, W) of every level, drawing exactly the xi a single
process would draw for those indices (the sample points are a counter-based
function of (seed, level, index)), and never exchanges data while solving.
The one exchange is at the end: every rank's per-sample level differences
Y_l = Q_l - Q_{l-1} are gathered to rank 0 in rank order, which is index
order, and the estimator of eq. StandardML runs over them in the library
(mlq_mlmc_combine, sums in index order).  The merged estimate is therefore
the single-process estimate of the same allocation, bit for bit.
"""
from __future__ import annotations

import numpy as np


def shard(n: int, rank: int, world: int):
    """The contiguous sample indices [first, first + count) of `rank`."""
    first = n * rank // world
    return first, n * (rank + 1) // world - first


def _device(group):
    """Tensors for collectives live on the GPU under NCCL, else on the host."""
    import torch
    import torch.distributed as dist

    if dist.get_backend(group) == "nccl":
        return torch.device("cuda", torch.cuda.current_device())
    return torch.device("cpu")


def gather_levels(ys_local, group=None):
    """Gather the per-level arrays ys_local[l] (1-D FP64) of every rank to
    rank 0.  Returns on rank 0 the per-level concatenation in rank order,
    elsewhere None."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    dev = _device(group)
    out = []
    for y in ys_local:
        y = np.ascontiguousarray(y, dtype=np.float64)
        n = torch.tensor([y.size], dtype=torch.int64, device=dev)
        sizes = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in range(world)]
        dist.all_gather(sizes, n, group=group)
        width = int(max(int(s.item()) for s in sizes))
        buf = torch.zeros(width, dtype=torch.float64, device=dev)
        buf[: y.size] = torch.from_numpy(y).to(dev)
        parts = [torch.zeros(width, dtype=torch.float64, device=dev) for _ in range(world)]
        dist.all_gather(parts, buf, group=group)
        if rank == 0:
            out.append(np.concatenate([p[: int(s.item())].cpu().numpy() for p, s in zip(parts, sizes)]))
    return out if rank == 0 else None


def combine_estimates(ys_local, group=None):
    """Rank-order merge of every rank's level differences and eq.
    StandardML over them (mlq_mlmc_combine); (estimate, V_l, RMSE_stat) on
    rank 0, None elsewhere."""
    from paper_2105_02007_gb300 import mlq

    ys = gather_levels(ys_local, group)
    return mlq.mlmc_combine(ys) if ys is not None else None


def max_over_ranks(x: float, group=None) -> float:
    """The maximum of x over the ranks (the job's time is its slowest rank's)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=_device(group))
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
