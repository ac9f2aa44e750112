"""Multi-rank host logic on CPU (gloo, two ranks): the rank-order merge of
per-sample level differences equals the single-process estimator over the
concatenated samples, and the job time is the slowest rank's."""
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
