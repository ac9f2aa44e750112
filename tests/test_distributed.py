"""Multi-rank host logic on CPU (gloo, two ranks): each rank takes the
contiguous sample range of one allocation, the rank-order merge of the
per-sample level differences through the library's estimator equals the
single-process estimate bit for bit, and the job time is the slowest rank's."""
import os
import socket

import numpy as np
import pytest

import oracle as O


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _levels(rank):
    rng = np.random.default_rng(100 + rank)
    # ragged per-rank sample counts on every level
    return [rng.normal(1e-3, 1e-4, 40 + 7 * rank), rng.normal(0, 1e-5, 9 + rank), rng.normal(0, 3e-6, 3 + 2 * rank)]


def _worker(rank, world, port, outdir):
    import torch.distributed as dist

    from paper_2105_02007_gb300 import distributed as D

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        res = D.combine_estimates(_levels(rank))
        t = D.max_over_ranks(1.5 + rank)
        if rank == 0:
            est, var, rmse = res
            np.save(os.path.join(outdir, "res.npy"), np.array([est, rmse, t] + list(var)))
        else:
            assert res is None
    finally:
        dist.destroy_process_group()


def test_two_rank_merge_matches_single_process(tmp_path):
    import torch.multiprocessing as mp

    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    got = np.load(tmp_path / "res.npy")
    ys = [np.concatenate([_levels(r)[l] for r in range(world)]) for l in range(3)]
    est, var, rmse = O.mlmc_estimate(ys)
    assert abs(got[0] - est) <= 1e-15 * abs(est)
    assert abs(got[1] - rmse) <= 1e-12 * rmse
    assert np.allclose(got[3:], var, rtol=1e-12, atol=0)
    assert got[2] == 2.5


def _full_levels():
    rng = np.random.default_rng(7)
    return [rng.normal(1e-3, 1e-4, 91), rng.normal(0, 1e-5, 17), rng.normal(0, 3e-6, 8)]


def _shard_worker(rank, world, port, outdir):
    import torch.distributed as dist

    from paper_2105_02007_gb300 import build

    build.build()
    from paper_2105_02007_gb300 import distributed as D

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = []
        for y in _full_levels():
            first, count = D.shard(y.size, rank, world)
            mine.append(y[first:first + count])
        res = D.combine_estimates(mine)
        if rank == 0:
            est, var, rmse = res
            np.save(os.path.join(outdir, "shard.npy"), np.array([est, rmse] + list(var)))
    finally:
        dist.destroy_process_group()


def test_two_rank_shards_equal_one_process_bit_for_bit(tmp_path):
    import torch.multiprocessing as mp

    from paper_2105_02007_gb300 import build

    build.build()
    from paper_2105_02007_gb300 import mlq

    world = 2
    mp.start_processes(_shard_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    got = np.load(tmp_path / "shard.npy")
    est, var, rmse = mlq.mlmc_combine(_full_levels())
    assert got[0] == est and got[1] == rmse and np.array_equal(got[2:], var)
    ref = O.mlmc_estimate(_full_levels())
    assert abs(est - ref[0]) <= 1e-15 * abs(ref[0]) and abs(rmse - ref[2]) <= 1e-12 * ref[2]


def test_shards_cover_the_allocation_and_draw_the_same_points():
    from paper_2105_02007_gb300 import distributed as D
    from paper_2105_02007_gb300 import inputs

    for n in (2, 16, 64, 1024, 4096):
        for world in (1, 2, 3, 8):
            parts = [D.shard(n, r, world) for r in range(world)]
            assert parts[0][0] == 0 and sum(c for _, c in parts) == n
            assert all(parts[r][0] + parts[r][1] == parts[r + 1][0] for r in range(world - 1))
    full = inputs.gaussian_xi(0, 3, 0, 64, 16)
    pieces = [inputs.gaussian_xi(0, 3, f, c, 16) for f, c in (D.shard(64, r, 3) for r in range(3))]
    assert np.array_equal(np.concatenate(pieces), full)
