"""Multi-rank combination of MLMC estimates (host side, torch.distributed).

Samples are independent, so N ranks run N replicas of an estimate on their
own draws (seed = rank) and never exchange data while solving.  The one
exchange is at the end: every rank's per-sample level differences
Y_l = Q_l - Q_{l-1} are gathered to rank 0 and the estimator of eq.
StandardML (sample means per level, unbiased sample variances, RMSE_stat =
sqrt(sum_l V_l / N_l)) is evaluated over all of them in rank order, so the
result does not depend on the order in which ranks finish.
"""
from __future__ import annotations

import numpy as np


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


def mlmc_from_levels(ys):
    """Estimate, per-level unbiased variances and RMSE_stat over the samples
    of each level (sums in index order)."""
    est, var, mse = 0.0, [], 0.0
    for y in ys:
        y = np.asarray(y, dtype=np.float64)
        n = y.size
        m = 0.0
        for v in y:
            m += float(v)
        m /= n
        s = 0.0
        for v in y:
            s += (float(v) - m) ** 2
        v_l = s / (n - 1) if n > 1 else 0.0
        est += m
        var.append(v_l)
        mse += v_l / n
    return est, var, mse ** 0.5


def combine_estimates(ys_local, group=None):
    """Rank-order merge of every rank's level differences; (estimate, V_l,
    RMSE_stat) on rank 0, None elsewhere."""
    ys = gather_levels(ys_local, group)
    return mlmc_from_levels(ys) if ys is not None else None


def max_over_ranks(x: float, group=None) -> float:
    """The maximum of x over the ranks (the job's time is its slowest rank's)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=_device(group))
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
