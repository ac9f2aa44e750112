"""CUDA path (through the C ABI) against the FP64 oracle on the same seeded
inputs.

Tolerances (relative, per-sample QoI):
  FP64 path  1e-10: both sides solve every time block to ||r|| <= 1e-13 ||b||;
             the QoI moves with the residual only through 1^T r (the block
             conserves m^T v up to the residual), so the two agree far below
             1e-10 unless a term is wrong.
  mixed path 1e-6:  FP32 inner solves inside FP64 refinement to 1e-12.
"""
import numpy as np
import pytest

import oracle as O
from paper_2105_02007_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 1: 1e-6}


@pytest.fixture(scope="module")
def mlq():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_02007_gb300 import build

    build.build()
    from paper_2105_02007_gb300 import mlq as m

    return m


def rel(a, b):
    return np.max(np.abs(np.asarray(a) - np.asarray(b)) / np.abs(np.asarray(b)))


# --------------------------------------------------------------------------
# C1: plain MC, 33 x 33 nodes, K = 16, 32 samples from seed 0, dt 0.05 x 200
# --------------------------------------------------------------------------
@pytest.fixture(scope="module")
def c1():
    mesh = O.mesh2d(33)
    modes, _ = O.kl_build(mesh, 0.09, 0.04, 16)
    phi = O.centroid_table(mesh, modes, mesh)
    xi = inputs.gaussian_xi(0, 0, 0, 32, 16)
    q, it, st = O.solve_batch(mesh, phi, xi, 0.05, 200)
    assert np.all(st == 0)
    return dict(mesh=mesh, phi=phi, xi=xi, q=q)


@pytest.mark.parametrize("precond", [0, 1])
@pytest.mark.parametrize("storage", [1, 2])
@pytest.mark.parametrize("prec", [0, 1])
def test_c1_full_config_parity(mlq, c1, prec, storage, precond):
    if prec == 0 and precond == 1:
        pytest.skip("the FP64 path uses Jacobi only")
    with mlq.Context(0, prec, storage=storage, precond=precond) as ctx:
        ctx.add_level(0, 33, 0.05, 200)
        ctx.set_kl(0, c1["phi"])
        r = ctx.solve(0, c1["xi"])
    assert np.all(r["status"] == 0)
    assert rel(r["q_fine"], c1["q"]) < TOL[prec]
    assert np.all(r["iters"] > 0)


def field_err(a, b):
    """max over nodes and samples of |a - b|, relative to max |b|."""
    return np.max(np.abs(np.asarray(a) - np.asarray(b))) / np.max(np.abs(np.asarray(b)))


@pytest.fixture(scope="module")
def c1_states(c1):
    q, V, W, st = O.solve_states(c1["mesh"], c1["phi"], c1["xi"], 0.05, 200)
    assert np.all(st == 0)
    return dict(q=q, v=V, w=W)


@pytest.mark.parametrize("prec,precond,storage", [(0, 0, 0), (0, 0, 2), (1, 0, 0), (1, 1, 0), (1, 0, 2)])
def test_c1_final_state_parity(mlq, c1, c1_states, prec, precond, storage):
    # the whole field v_h(T) (and w(T)) node by node, not only Q = m^T v: a
    # wrong stencil entry, load or reaction term that leaves the integral
    # nearly unchanged still moves the field
    with mlq.Context(0, prec, storage=storage, precond=precond) as ctx:
        ctx.add_level(0, 33, 0.05, 200)
        ctx.set_kl(0, c1["phi"])
        r = ctx.solve_state(0, c1["xi"])
    assert np.all(r["status"] == 0)
    assert field_err(r["v"], c1_states["v"]) < TOL[prec]
    assert field_err(r["w"], c1_states["w"]) < TOL[prec]
    assert rel(r["q"], c1_states["q"]) < TOL[prec]


# --------------------------------------------------------------------------
# Launch shapes: cluster sizes 1..16 with ragged row bands, block sizes,
# random initial states (every node active), a mean angle field.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("storage", [1, 2])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("m,cluster,threads", [(17, 1, 64), (17, 2, 128), (17, 4, 96), (23, 8, 64),
                                               (33, 16, 128), (9, 4, 64)])
def test_launch_shapes_random_state(mlq, prec, m, cluster, threads, storage):
    mesh = O.mesh2d(m)
    rng = np.random.default_rng(m * 100 + cluster)
    K = 6
    modes, _ = O.kl_build(mesh, 0.09, 0.04, K)
    phi = O.centroid_table(mesh, modes, mesh)
    tm = rng.normal(scale=0.3, size=mesh.ne)
    v0 = rng.uniform(0, 1, size=mesh.n)
    w0 = rng.uniform(0, 0.2, size=mesh.n)
    xi = inputs.gaussian_xi(3, 0, 0, 5, K)
    q_ref, _, st = O.solve_batch(mesh, phi, xi, 0.1, 15, v0=v0, w0=w0, theta_mean=tm)
    assert np.all(st == 0)
    try:
        ctx = mlq.Context(0, prec, cluster=cluster, threads=threads, storage=storage, precond=0)
    except mlq.MLQError as e:
        if e.code == -6:
            pytest.skip("cluster size not available on this device")
        raise
    with ctx:
        ctx.add_level(0, m, 0.1, 15)
        ctx.set_kl(0, phi, tm)
        ctx.set_initial_state(0, v0, w0)
        c_, t_, res_ = ctx.level_launch(0, True)
        assert (c_, t_) == (cluster, threads) and (res_ > 0) == (storage == 1)
        r = ctx.solve(0, xi)
    assert np.all(r["status"] == 0)
    assert rel(r["q_fine"], q_ref) < TOL[prec]


# --------------------------------------------------------------------------
# Multilevel pairs: Y = Q_l - Q_{l-1} with the same xi on both members,
# Phi transferred from the finest mesh by the midpoint rule.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("prec", [0, 1])
def test_level_pair_and_telescoping(mlq, prec):
    ms, dts = [9, 17, 33], [0.2, 0.1, 0.05]
    T = 4.0
    fine = O.mesh2d(33)
    modes, _ = O.kl_build(fine, 0.09, 0.04, 8)
    meshes = [O.mesh2d(m) for m in ms]
    phis = [O.centroid_table(fine, modes, mm) for mm in meshes]
    xi = inputs.gaussian_xi(0, 2, 0, 6, 8)
    qref = [O.solve_batch(mm, ph, xi, dt, int(round(T / dt)))[0] for mm, ph, dt in zip(meshes, phis, dts)]
    with mlq.Context(0, prec) as ctx:
        for l, (m, dt, ph) in enumerate(zip(ms, dts, phis)):
            ctx.add_level(l, m, dt, int(round(T / dt)))
            ctx.set_kl(l, ph)
        r2 = ctx.solve(2, xi, with_coarse=True)
        r1 = ctx.solve(1, xi, with_coarse=True)
        r0 = ctx.solve(0, xi)
    assert rel(r2["q_fine"], qref[2]) < TOL[prec]
    assert rel(r2["q_coarse"], qref[1]) < TOL[prec]
    assert rel(r1["q_coarse"], qref[0]) < TOL[prec]
    # the coarse member of pair l is the fine member of pair l-1, bit for bit
    assert np.array_equal(r2["q_coarse"], r1["q_fine"])
    assert np.array_equal(r1["q_coarse"], r0["q_fine"])
    assert np.array_equal(r2["y"], r2["q_fine"] - r2["q_coarse"])
    tele = r0["y"] + r1["y"] + r2["y"]
    assert np.allclose(tele, r2["q_fine"], rtol=1e-14, atol=0)


# --------------------------------------------------------------------------
# Edge cases
# --------------------------------------------------------------------------
@pytest.mark.parametrize("prec", [0, 1])
def test_edge_cases(mlq, prec):
    # smallest mesh (2 x 2 nodes), one sample, zero steps (Q = m^T v0)
    mesh = O.mesh2d(2)
    rng = np.random.default_rng(0)
    v0 = rng.uniform(0, 1, 4)
    with mlq.Context(0, prec) as ctx:
        ctx.add_level(0, 2, 0.1, 0)
        ctx.set_kl(0, np.ones((2, 1)))
        ctx.set_initial_state(0, v0)
        r = ctx.solve(0, np.zeros((1, 1)))
        mlump = np.array([2, 1, 1, 2]) / 6.0
        assert abs(r["q_fine"][0] - mlump @ v0) < 1e-15
        ctx.add_level(0, 2, 0.1, 7)
        ctx.set_kl(0, np.ones((2, 1)))
        ctx.set_initial_state(0, v0)
        r = ctx.solve(0, np.array([[0.3], [-1.2]]))
    qref = O.solve_batch(mesh, np.ones((2, 1)), np.array([[0.3], [-1.2]]), 0.1, 7, v0=v0)[0]
    assert rel(r["q_fine"], qref) < TOL[prec]
    # an empty batch is a no-op
    with mlq.Context(0, prec) as ctx:
        ctx.add_level(0, 9, 0.1, 3)
        ctx.set_kl(0, np.zeros((128, 2)))
        r = ctx.solve(0, np.zeros((0, 2)))
        assert r["q_fine"].size == 0


@pytest.mark.parametrize("prec", [0, 1])
def test_failures_are_per_sample(mlq, prec):
    mesh = O.mesh2d(17)
    modes, _ = O.kl_build(mesh, 0.09, 0.04, 4)
    phi = O.centroid_table(mesh, modes, mesh)
    xi = inputs.gaussian_xi(0, 0, 0, 4, 4)
    bad = xi.copy()
    bad[2, 1] = np.nan
    with mlq.Context(0, prec) as ctx:
        ctx.add_level(0, 17, 0.1, 10)
        ctx.set_kl(0, phi)
        good = ctx.solve(0, xi)
        mixed = ctx.solve(0, bad)
        assert mixed["status"][2] == 2 and np.isnan(mixed["q_fine"][2])
        keep = [0, 1, 3]
        assert np.array_equal(mixed["q_fine"][keep], good["q_fine"][keep])
        assert np.all(mixed["status"][keep] == 0)
        # an iteration cap of 1 is reported, and the sample still finishes
        ctx.set_options(max_iter=1, max_sweeps=1)
        capped = ctx.solve(0, xi)
        assert np.all(capped["status"] == 1) and np.all(np.isfinite(capped["q_fine"]))


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_invariance(mlq, prec):
    mesh = O.mesh2d(33)
    modes, _ = O.kl_build(mesh, 0.09, 0.04, 8)
    phi = O.centroid_table(mesh, modes, mesh)
    xi = inputs.gaussian_xi(0, 0, 0, 40, 8)
    with mlq.Context(0, prec) as ctx:
        ctx.add_level(0, 33, 0.1, 20)
        ctx.set_kl(0, phi)
        full = ctx.solve(0, xi)
        part = ctx.solve(0, xi[17:21])
        one = ctx.solve(0, xi[30:31])
    assert np.array_equal(full["q_fine"][17:21], part["q_fine"])
    assert np.array_equal(full["q_fine"][30:31], one["q_fine"])


def test_device_tensors_in_and_out(mlq):
    import torch

    mesh = O.mesh2d(17)
    modes, _ = O.kl_build(mesh, 0.09, 0.04, 4)
    phi = O.centroid_table(mesh, modes, mesh)
    xi = inputs.gaussian_xi(0, 0, 0, 8, 4)
    with mlq.Context(0, 0) as ctx:
        ctx.add_level(0, 17, 0.1, 10)
        ctx.set_kl(0, phi)
        host = ctx.solve(0, xi)
        dxi = torch.from_numpy(xi).cuda()
        out = dict(q_fine=torch.zeros(8, dtype=torch.float64, device="cuda"),
                   status=torch.zeros(8, dtype=torch.int32, device="cuda"))
        ctx.solve(0, dxi, out=out)
        torch.cuda.synchronize()
    assert np.array_equal(out["q_fine"].cpu().numpy(), host["q_fine"])


# --------------------------------------------------------------------------
# Full-size meshes of the MLMC hierarchy in the launch shapes the benchmark
# uses: 257 x 257 and 129 x 129 nodes at their time steps, over a window of
# time blocks the oracle finishes in seconds, on sampled xi.
# --------------------------------------------------------------------------
@pytest.fixture(scope="module")
def modes257():
    fine = O.mesh2d(257)
    return fine, O.kl_build(fine, 0.09, 0.04, 16)[0]


@pytest.mark.parametrize("storage", [0, 2])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("m,dt", [(129, 0.0125), (257, 0.00625)])
def test_full_size_meshes_sampled(mlq, modes257, prec, m, dt, storage):
    # 12 blocks at 257 x 257: the multigrid path's extrapolated initial guess
    # reaches its full order (4) from block 9 on, so the window covers it
    steps = 12 if m == 257 else 16
    fine, modes = modes257
    mesh = fine if m == 257 else O.mesh2d(m)
    phi = O.centroid_table(fine, modes, mesh)
    xi = inputs.gaussian_xi(0, 4, 0, 2, 16)
    q_ref, V_ref, W_ref, st = O.solve_states(mesh, phi, xi, dt, steps)
    assert np.all(st == 0)
    with mlq.Context(0, prec, storage=storage) as ctx:
        ctx.add_level(0, m, dt, steps)
        ctx.set_kl(0, phi)
        r = ctx.solve(0, xi)
        f = ctx.solve_state(0, xi)
    assert np.all(r["status"] == 0)
    assert rel(r["q_fine"], q_ref) < TOL[prec]
    assert np.array_equal(f["q"], r["q_fine"])
    assert field_err(f["v"], V_ref) < TOL[prec]
    assert field_err(f["w"], W_ref) < TOL[prec]


@pytest.mark.parametrize("prec", [0, 1])
def test_full_size_conservation_and_uniform_state(mlq, prec):
    # properties that hold at any size: one block conserves m^T (v + dt R);
    # a spatially constant state follows the scalar recurrence.
    m, dt = 257, 0.00625
    rng = np.random.default_rng(1)
    fine = O.mesh2d(257)
    phi = rng.normal(scale=0.2, size=(fine.ne, 4))
    xi = inputs.gaussian_xi(0, 4, 0, 4, 4)
    v0 = rng.uniform(0, 1, size=fine.n)
    w0 = rng.uniform(0, 0.2, size=fine.n)
    rp, ci, mv, _ = O.assemble(fine)
    mvec = np.zeros(fine.n)
    np.add.at(mvec, ci, mv)
    R = v0 * (v0 - 0.1) * (1 - v0) - w0
    expect = mvec @ (v0 + dt * R)
    with mlq.Context(0, prec) as ctx:
        ctx.add_level(0, m, dt, 1)
        ctx.set_kl(0, phi)
        ctx.set_initial_state(0, v0, w0)
        r = ctx.solve(0, xi)
        assert np.all(np.abs(r["q_fine"] - expect) < TOL[prec] * abs(expect))
        ctx.add_level(0, m, dt, 50)
        ctx.set_kl(0, phi)
        ctx.set_initial_state(0, np.full(fine.n, 0.6), np.full(fine.n, 0.05))
        r = ctx.solve(0, xi)
    v, w = 0.6, 0.05
    for _ in range(50):
        v, w = v + dt * (v * (v - 0.1) * (1 - v) - w), w + dt * 0.01 * (v - 0.5 * w)
    assert np.all(np.abs(r["q_fine"] - v) < (1e-12 if prec == 0 else 1e-7) * v)


# --------------------------------------------------------------------------
# MLMC estimator through the C ABI against the oracle's estimator on the
# per-sample values it computes (small hierarchy).
# --------------------------------------------------------------------------
@pytest.mark.parametrize("prec", [0, 1])
def test_mlmc_estimate_matches_oracle(mlq, prec):
    ms, dts, N = [9, 17, 33], [0.2, 0.1, 0.05], [40, 12, 4]
    T = 2.0
    fine = O.mesh2d(33)
    modes, _ = O.kl_build(fine, 0.09, 0.04, 8)
    meshes = [O.mesh2d(m) for m in ms]
    phis = [O.centroid_table(fine, modes, mm) for mm in meshes]
    xis = [inputs.gaussian_xi(0, l, 0, N[l], 8) for l in range(3)]
    yref = []
    for l in range(3):
        qf = O.solve_batch(meshes[l], phis[l], xis[l], dts[l], int(round(T / dts[l])))[0]
        if l == 0:
            yref.append(qf)
        else:
            qc = O.solve_batch(meshes[l - 1], phis[l - 1], xis[l], dts[l - 1], int(round(T / dts[l - 1])))[0]
            yref.append(qf - qc)
    est_ref, var_ref, rmse_ref = O.mlmc_estimate(yref)
    with mlq.Context(0, prec) as ctx:
        for l, (m, dt, ph) in enumerate(zip(ms, dts, phis)):
            ctx.add_level(l, m, dt, int(round(T / dt)))
            ctx.set_kl(l, ph)
        mean, var, rmse, ys = ctx.estimate(xis, return_y=True)
    tol = TOL[prec]
    assert abs(mean - est_ref) < tol * abs(est_ref)
    for l in range(3):
        assert np.max(np.abs(ys[l] - yref[l])) < tol * np.max(np.abs(yref[0]))
    assert abs(rmse - rmse_ref) < (1e-2 if prec else 1e-6) * rmse_ref


@pytest.mark.parametrize("precond", [0, 1])
@pytest.mark.parametrize("m", [17, 65])
def test_autotune_keeps_parity(mlq, m, precond):
    mesh = O.mesh2d(m)
    modes, _ = O.kl_build(mesh, 0.09, 0.04, 6)
    phi = O.centroid_table(mesh, modes, mesh)
    xi = inputs.gaussian_xi(5, 0, 0, 6, 6)
    q_ref = O.solve_batch(mesh, phi, xi, 0.05, 6)[0]
    with mlq.Context(0, 1, precond=precond) as ctx:
        ctx.add_level(0, m, 0.05, 6)
        ctx.set_kl(0, phi)
        cs, th, ms = ctx.autotune(0, xi, probe_steps=2)
        assert cs >= 1 and th >= 32 and ms > 0
        assert ctx.level_launch(0) == (cs, th)
        r = ctx.solve(0, xi)
    assert np.all(r["status"] == 0)
    assert rel(r["q_fine"], q_ref) < TOL[1]


# --------------------------------------------------------------------------
# KL synthesis step alone (row a2): FP64 CUDA-core path and the tcgen05
# tensor-core path of the mixed precision (TF32 split, FP32 accumulation),
# over ragged element and sample tiles and K padded to a multiple of 8.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("m,K,S", [(17, 16, 5), (17, 6, 300), (65, 16, 33), (33, 64, 17), (9, 1, 1)])
def test_kl_synthesis_parity(mlq, m, K, S):
    rng = np.random.default_rng(m * 1000 + K * 10 + S)
    ne = 2 * (m - 1) ** 2
    phi = rng.normal(scale=0.3 / np.sqrt(K), size=(ne, K))
    tm = rng.normal(scale=0.2, size=ne)
    xi = inputs.gaussian_xi(2, 1, 0, S, K)
    ref = O.kl_synthesis(phi, xi, tm)
    # Tensor-core bound: each TF32 part keeps 11 significant bits, so the
    # three-product split loses at most ~3 * 2^-20 |phi xi| per term (the
    # dropped lo*lo product and the truncation of both lo parts); FP32
    # accumulation of K terms adds K * 2^-24 sum |phi xi|; the argument of
    # cos/sin is 2 theta; sincosf and the FP32 rounding of theta add ~1e-6.
    l1 = np.max(np.abs(xi) @ np.abs(phi).T)
    tol_tc = 2 * (3 * 2.0 ** -20 + K * 2.0 ** -24) * l1 + 1e-6
    for prec, tol in ((0, 1e-13), (1, tol_tc)):
        with mlq.Context(0, prec) as ctx:
            ctx.add_level(0, m, 0.1, 1)
            ctx.set_kl(0, phi, tm)
            got = ctx.synthesize(0, xi)
        assert np.max(np.abs(got - ref)) < tol, (prec, np.max(np.abs(got - ref)))


def test_estimate_graph_capture_and_replay(mlq):
    import torch

    ms, dts, N = [9, 17], [0.2, 0.1], [24, 8]
    fine = O.mesh2d(17)
    modes, _ = O.kl_build(fine, 0.09, 0.04, 4)
    phis = [O.centroid_table(fine, modes, O.mesh2d(m)) for m in ms]
    xis = [inputs.gaussian_xi(0, l, 0, N[l], 4) for l in range(2)]
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    d_xi = [torch.from_numpy(x).to(dev) for x in xis]
    res = {}
    for graphs in (0, 1):
        with mlq.Context(0, mlq.MLQ_MIXED, stream=stream.cuda_stream, graphs=graphs) as ctx:
            for l, (m, dt) in enumerate(zip(ms, dts)):
                ctx.add_level(l, m, dt, int(round(2.0 / dt)))
                ctx.set_kl(l, phis[l])
            torch.cuda.synchronize(dev)
            first = ctx.estimate(d_xi)
            n1 = ctx.launch_count()
            second = ctx.estimate(d_xi)                # replay when graphs = 1
            assert ctx.launch_count() == 2 * n1
            assert first[0] == second[0] and np.array_equal(first[1], second[1])
            # new values behind the same pointers are picked up by the replay
            d_xi[1].copy_(torch.from_numpy(inputs.gaussian_xi(1, 1, 0, N[1], 4)).to(dev))
            third = ctx.estimate(d_xi)
            d_xi[1].copy_(torch.from_numpy(xis[1]).to(dev))
            res[graphs] = (first, third)
    assert res[0][0][0] == res[1][0][0]
    assert res[0][1][0] == res[1][1][0] and res[0][1][0] != res[0][0][0]


# --------------------------------------------------------------------------
# Multigrid-preconditioned inner PCG (mixed path): same QoI as the oracle,
# on every cluster size that fits, over the nested hierarchy of each mesh.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("m,cluster,steps", [(3, 1, 5), (9, 1, 6), (9, 8, 5), (17, 1, 10), (17, 4, 6),
                                             (17, 16, 6), (33, 2, 8), (33, 16, 5), (65, 1, 6), (65, 4, 6),
                                             (129, 4, 4), (129, 16, 3), (257, 16, 3)])
def test_multigrid_parity(mlq, m, cluster, steps):
    mesh = O.mesh2d(m)
    rng = np.random.default_rng(m + cluster)
    K = 6
    modes, _ = O.kl_build(mesh, 0.09, 0.04, K)
    phi = O.centroid_table(mesh, modes, mesh)
    v0 = rng.uniform(0, 1, size=mesh.n)
    w0 = rng.uniform(0, 0.2, size=mesh.n)
    dt = 0.1 * 16.0 / (m - 1)
    xi = inputs.gaussian_xi(4, 0, 0, 3, K)
    q_ref, _, st = O.solve_batch(mesh, phi, xi, dt, steps, v0=v0, w0=w0, nthreads=2)
    assert np.all(st == 0)
    try:
        ctx = mlq.Context(0, mlq.MLQ_MIXED, precond=1, cluster=cluster)
    except mlq.MLQError as e:
        if e.code == -6:
            pytest.skip("cluster size not available")
        raise
    with ctx:
        ctx.add_level(0, m, dt, steps)
        ctx.set_kl(0, phi)
        ctx.set_initial_state(0, v0, w0)
        assert ctx.level_launch(0, True)[2] == 3
        r = ctx.solve(0, xi)
    assert np.all(r["status"] == 0), r["status"]
    assert rel(r["q_fine"], q_ref) < TOL[1]


# --------------------------------------------------------------------------
# The paper's QMC variant: Halton points (from point 1, skipping the origin)
# mapped to the uniform KL variables xi = sqrt(3)(2y - 1), through the solver.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("prec", [0, 1])
def test_halton_uniform_points_parity(mlq, prec):
    m, K, S, dt, nsteps = 33, 8, 16, 0.05, 40
    mesh = O.mesh2d(m)
    modes, _ = O.kl_build(mesh, 0.09, 0.04, K)
    phi = O.centroid_table(mesh, modes, mesh)
    xi = inputs.uniform_xi(inputs.halton(S, K, first=1))
    assert np.max(np.abs(xi)) < np.sqrt(3.0)
    q_ref, _, st = O.solve_batch(mesh, phi, xi, dt, nsteps, nthreads=2)
    assert np.all(st == 0)
    with mlq.Context(0, prec) as ctx:
        ctx.add_level(0, m, dt, nsteps)
        ctx.set_kl(0, phi)
        r = ctx.solve(0, xi)
    assert np.all(r["status"] == 0)
    assert rel(r["q_fine"], q_ref) < TOL[prec]
