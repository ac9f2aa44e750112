"""Serving (mlq_submit / mlq_poll): requests for the Monte Carlo mean of Q_l,
answered by the context's batching worker, against direct batched solves
of the same samples.

A request stops at the first chunk boundary n (a multiple of its chunk, or
all samples) where sqrt(V_n / n) <= target; each sample's Q depends only on
its own xi, so the served mean over the first n samples equals the mean of
the same n values from one direct solve, bit for bit on 2D levels.
"""
import numpy as np
import pytest

import oracle as O
from paper_2105_02007_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mlq():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_02007_gb300 import build

    build.build()
    from paper_2105_02007_gb300 import mlq as m

    return m


LEVELS = [(9, 0.1, 10), (17, 0.05, 20)]   # m, dt, blocks
K = 4


def make_ctx(mlq):
    ctx = mlq.Context(0, mlq.MLQ_MIXED)
    fine = O.mesh2d(17)
    modes, _ = O.kl_build(fine, 0.09, 0.04, K)
    for l, (m, dt, n) in enumerate(LEVELS):
        ctx.add_level(l, m, dt, n)
        ctx.set_kl(l, O.centroid_table(fine, modes, O.mesh2d(m)))
    return ctx


def expected(q, target, chunk):
    """(n, mean, rmse) of the stopping rule applied to values in index order
    (sums accumulated one value after another, as the library does)."""
    S = len(q)
    b = 0
    while True:
        b = min(b + chunk, S)
        mean = 0.0
        for x in q[:b]:
            mean += float(x)
        mean /= b
        var = 0.0
        for x in q[:b]:
            var += (float(x) - mean) * (float(x) - mean)
        rmse = float(np.sqrt(var / (b - 1) / b)) if b > 1 else np.inf
        if (target > 0 and b >= 2 and rmse <= target) or b == S:
            return b, mean, rmse


def test_serve_matches_direct_solves_and_stopping_rule(mlq):
    reqs = [(0, 200, 3e-5, 16, 1), (1, 64, 1e-4, 8, 2), (0, 37, 0.0, 16, 3), (1, 100, 5e-6, 32, 4),
            (0, 1, 1e-3, 16, 5), (1, 40, 1.0, 4, 6)]
    with make_ctx(mlq) as ctx:
        xis = [inputs.gaussian_xi(seed, lvl, 0, S, K) for lvl, S, _, _, seed in reqs]
        tickets = [ctx.submit(lvl, xi, tgt, ch) for (lvl, S, tgt, ch, _), xi in zip(reqs, xis)]
        results = [ctx.wait(t) for t in tickets]
        for (lvl, S, tgt, ch, _), xi, r in zip(reqs, xis, results):
            assert r["status"] == 0 and r["worst"] == 0
            q = ctx.solve(lvl, xi)["q_fine"]
            n, mean, rmse = expected(q, tgt, ch)
            assert r["samples_used"] == n
            assert r["mean"] == mean
            if n > 1:
                assert abs(r["rmse"] - rmse) <= 1e-15 * rmse
            assert r["batches"] >= 1 and r["latency_ms"] > 0
        # a released ticket is gone
        with pytest.raises(mlq.MLQError):
            ctx.poll(tickets[0])


def test_serve_result_does_not_depend_on_the_mix(mlq):
    xi = inputs.gaussian_xi(9, 1, 0, 96, K)
    with make_ctx(mlq) as ctx:
        alone = ctx.wait(ctx.submit(1, xi, 2e-5, 16))
    with make_ctx(mlq) as ctx:
        others = [ctx.submit(l, inputs.gaussian_xi(20 + l, l, 0, 50, K), 1e-5, 8) for l in (0, 1, 0)]
        t = ctx.submit(1, xi, 2e-5, 16)
        more = [ctx.submit(1, inputs.gaussian_xi(30, 1, 0, 70, K), 0.0, 16)]
        mixed = ctx.wait(t)
        for o in others + more:
            assert ctx.wait(o)["status"] == 0
    for k in ("samples_used", "mean", "rmse", "worst", "status"):
        assert alone[k] == mixed[k], k


def test_serve_3d_level(mlq):
    dims = (9, 9, 5)
    mesh = O.mesh3d(*dims)
    modes, _ = O.kl_build(mesh, 0.09, 0.15 ** 2, K)
    xi = inputs.gaussian_xi(4, 0, 0, 24, K)
    with mlq.Context(0, mlq.MLQ_MIXED) as ctx:
        ctx.add_level(0, dims, 0.05, 6)
        ctx.set_kl(0, O.centroid_table(mesh, modes, mesh))
        r = ctx.wait(ctx.submit(0, xi, 0.0, 8))
        q = ctx.solve(0, xi)["q_fine"]
    assert r["status"] == 0 and r["samples_used"] == 24
    # the 3D launch shape follows the batch size: equal to rounding
    assert abs(r["mean"] - q.mean()) <= 1e-12 * abs(q.mean())


def test_serve_general_mesh_level_beside_a_structured_one(mlq):
    # a level on a general tetrahedral mesh (the shell) and a structured 2D
    # level in one context: requests on both are served together and each
    # mean equals the direct solves' (the launch shape follows the batch
    # size: equal to rounding)
    from paper_2105_02007_gb300 import lv_inputs as LV

    xyz, conn = LV.lv_mesh(2, 8, 14)
    frames, alpha = LV.lv_fibres(xyz, conn)
    rng = np.random.default_rng(73)
    phi = rng.normal(scale=0.3, size=(conn.shape[0], K))
    v0, w0 = LV.stimulus(xyz, radius=0.4)
    fine = O.mesh2d(17)
    modes, _ = O.kl_build(fine, 0.09, 0.04, K)
    xs = inputs.gaussian_xi(46, 0, 0, 40, K)
    xm = inputs.gaussian_xi(47, 1, 0, 24, K)
    with mlq.Context(0, mlq.MLQ_MIXED) as ctx:
        ctx.add_level(0, 17, 0.05, 20)
        ctx.set_kl(0, O.centroid_table(fine, modes, fine))
        ctx.add_level_mesh(1, xyz, conn, 0.05, 8, frames=frames)
        ctx.set_kl(1, phi, alpha)
        ctx.set_initial_state(1, v0, w0)
        tm = ctx.submit(1, xm, 0.0, 8)
        ts = ctx.submit(0, xs, 0.0, 8)
        rm, rs = ctx.wait(tm), ctx.wait(ts)
        qm = ctx.solve(1, xm)["q_fine"]
        qs = ctx.solve(0, xs)["q_fine"]
    assert rm["status"] == 0 and rs["status"] == 0
    assert rm["samples_used"] == 24 and rs["samples_used"] == 40
    assert abs(rm["mean"] - qm.mean()) <= 1e-10 * abs(qm.mean())
    assert abs(rs["mean"] - qs.mean()) <= 1e-10 * abs(qs.mean())


def test_serve_rejects_bad_requests(mlq):
    with make_ctx(mlq) as ctx:
        xi = inputs.gaussian_xi(1, 0, 0, 8, K)
        for bad in (dict(level=5), dict(chunk=3)):
            args = dict(level=0, xi=xi, target_rmse=0.0, chunk=8)
            args.update(bad)
            with pytest.raises(mlq.MLQError):
                ctx.submit(**args)
        with pytest.raises(mlq.MLQError):
            ctx.poll(12345)


# --------------------------------------------------------------------------
# Continuous batching across levels and admission by device memory
# --------------------------------------------------------------------------
MIX = [(33, 0.05, 200), (65, 0.025, 400)]   # two levels whose batches run for a while


def make_mix_ctx(mlq):
    ctx = mlq.Context(0, mlq.MLQ_MIXED)
    fine = O.mesh2d(65)
    modes, _ = O.kl_build(fine, 0.09, 0.04, K)
    for l, (m, dt, n) in enumerate(MIX):
        ctx.add_level(l, m, dt, n)
        ctx.set_kl(l, O.centroid_table(fine, modes, O.mesh2d(m)))
    return ctx


def overlap(a, b):
    return min(a["last_ms"], b["last_ms"]) - max(a["first_ms"], b["first_ms"])


def test_serve_levels_run_together_and_results_unchanged(mlq):
    xa = inputs.gaussian_xi(41, 0, 0, 64, K)
    xb = inputs.gaussian_xi(42, 1, 0, 32, K)
    with make_mix_ctx(mlq) as ctx:
        ta = ctx.submit(0, xa, 0.0, 64)
        tb = ctx.submit(1, xb, 0.0, 32)
        ra, rb = ctx.wait(ta), ctx.wait(tb)
        qa = ctx.solve(0, xa)["q_fine"]
        qb = ctx.solve(1, xb)["q_fine"]
    assert ra["status"] == 0 and rb["status"] == 0
    assert ra["batches"] == 1 and rb["batches"] == 1
    assert overlap(ra, rb) > 0                 # the two levels were on the device together
    n, mean, _ = expected(qa, 0.0, 64)
    assert ra["mean"] == mean and ra["samples_used"] == 64
    n, mean, _ = expected(qb, 0.0, 32)
    assert rb["mean"] == mean and rb["samples_used"] == 32


def test_serve_waits_for_memory_and_refuses_what_never_fits(mlq):
    xa = inputs.gaussian_xi(43, 0, 0, 64, K)
    xb = inputs.gaussian_xi(44, 1, 0, 32, K)
    with make_mix_ctx(mlq) as ctx:
        ba, bb = ctx.workspace_bytes(0, 64), ctx.workspace_bytes(1, 32)
        # room for either batch, not for both: the second waits for the first
        ctx.serve_limits(6, max(ba, bb) + 4096)
        ta = ctx.submit(0, xa, 0.0, 64)
        tb = ctx.submit(1, xb, 0.0, 32)
        ra, rb = ctx.wait(ta), ctx.wait(tb)
        assert ra["status"] == 0 and rb["status"] == 0
        assert overlap(ra, rb) <= 0
        alone_a = ctx.solve(0, xa)["q_fine"]
        assert ra["mean"] == expected(alone_a, 0.0, 64)[1]
        # a budget below one batch: the request is refused, the next one served
        ctx.serve_limits(6, min(ba, bb) // 4)
        r = ctx.wait(ctx.submit(1, xb, 0.0, 32))
        assert r["status"] == mlq.MLQ_ENOMEM and r["samples_used"] == 0
        ctx.serve_limits(6, 0)
        r2 = ctx.wait(ctx.submit(1, xb, 0.0, 32))
        assert r2["status"] == 0 and r2["mean"] == rb["mean"]
