"""3D levels (P1 on Kuhn tetrahedra of the box [0,1]^2 x [0,0.25]) through
the C ABI against the FP64 oracle on the same seeded inputs.

Tolerances as for 2D (relative, per-sample QoI): FP64 path 1e-10, mixed path
1e-6 (FP32 inner PCG inside FP64 refinement to 1e-12); the QoI moves with the
solver only through 1^T r, the residual of each block.
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


def setup3d(dims, K, seed, S, radius=0.29):
    mesh = O.mesh3d(*dims)
    modes, _ = O.kl_build(mesh, 0.09, 0.15 ** 2, K)
    phi = O.centroid_table(mesh, modes, mesh)
    xi = inputs.gaussian_xi(seed, 0, 0, S, K)
    v0, w0 = O.initial_state(mesh, radius)
    return mesh, phi, xi, v0, w0


# every built cluster size (a CTA may own no grid line: 9 x 7 x 5 on 8),
# 20 and 24 CTAs per sample in one cooperative launch (global barriers),
# ragged line bands, rows padded from 5, 9, 13, 17, 33 to multiples of 4, FP64 and the
# mixed path with the Jacobi and the multigrid inner preconditioner (meshes
# with 1..4 multigrid levels; 13 x 11 x 6 cannot be coarsened)
@pytest.mark.parametrize("dims,cluster", [((5, 5, 3), 1), ((9, 9, 5), 1), ((9, 9, 5), 4), ((9, 7, 5), 8),
                                          ((17, 17, 5), 16), ((17, 17, 5), 12), ((13, 11, 6), 2),
                                          ((13, 11, 6), 6), ((33, 33, 9), 4), ((17, 17, 5), 20),
                                          ((33, 33, 9), 24)])
@pytest.mark.parametrize("prec,precond", [(0, 0), (1, 0), (1, 1)])
def test_3d_parity(mlq, dims, cluster, prec, precond):
    mesh, phi, xi, v0, w0 = setup3d(dims, 6, 11, 5)
    nsteps, dt = 8, 0.05
    q_ref, _, st = O.solve_batch(mesh, phi, xi, dt, nsteps, v0=v0, w0=w0, nthreads=2)
    assert np.all(st == 0)
    try:
        ctx = mlq.Context(0, prec, cluster=cluster, precond=precond)
    except mlq.MLQError as e:
        if e.code == -6:
            pytest.skip("cluster size not available")
        raise
    with ctx:
        ctx.add_level(0, dims, dt, nsteps)
        ctx.set_kl(0, phi)
        ctx.set_initial_disk(0, 0.29)   # no node on the sphere of any mesh here
        assert ctx.level_launch(0)[0] == cluster
        r = ctx.solve(0, xi)
    assert np.all(r["status"] == 0), r["status"]
    assert rel(r["q_fine"], q_ref) < TOL[prec]


@pytest.mark.parametrize("dims,cluster", [((9, 9, 5), 1), ((17, 17, 5), 4), ((33, 33, 9), 4), ((33, 33, 9), 24)])
@pytest.mark.parametrize("prec,precond", [(0, 0), (1, 0), (1, 1)])
def test_3d_final_state_parity(mlq, dims, cluster, prec, precond):
    # the field v_h(T), w(T) node by node against the oracle (relative to max |v|)
    mesh, phi, xi, v0, w0 = setup3d(dims, 6, 13, 3)
    nsteps, dt = 10, 0.05
    q_ref, V, W, st = O.solve_states(mesh, phi, xi, dt, nsteps, v0=v0, w0=w0)
    assert np.all(st == 0)
    with mlq.Context(0, prec, cluster=cluster, precond=precond) as ctx:
        ctx.add_level(0, dims, dt, nsteps)
        ctx.set_kl(0, phi)
        ctx.set_initial_disk(0, 0.29)
        r = ctx.solve_state(0, xi)
    assert np.all(r["status"] == 0), r["status"]
    assert rel(r["q"], q_ref) < TOL[prec]
    assert np.max(np.abs(r["v"] - V)) / np.max(np.abs(V)) < TOL[prec]
    assert np.max(np.abs(r["w"] - W)) / np.max(np.abs(W)) < TOL[prec]


@pytest.mark.parametrize("prec", [0, 1])
def test_3d_random_state_and_lengths(mlq, prec):
    # a non-default box and a random initial state (every stencil entry and
    # the reaction matter), more blocks
    dims, lengths = (9, 6, 4), (1.0, 0.6, 0.3)
    mesh = O.mesh3d(*dims, *lengths)
    modes, _ = O.kl_build(mesh, 0.09, 0.04, 5)
    phi = O.centroid_table(mesh, modes, mesh)
    rng = np.random.default_rng(3)
    v0 = rng.uniform(0, 1, mesh.n)
    w0 = rng.uniform(0, 0.2, mesh.n)
    xi = inputs.gaussian_xi(5, 0, 0, 4, 5)
    q_ref, _, st = O.solve_batch(mesh, phi, xi, 0.02, 20, v0=v0, w0=w0, nthreads=2)
    assert np.all(st == 0)
    with mlq.Context(0, prec) as ctx:
        ctx.add_level(0, dims, 0.02, 20, lengths=lengths)
        ctx.set_kl(0, phi)
        ctx.set_initial_state(0, v0, w0)
        r = ctx.solve(0, xi)
    assert np.all(r["status"] == 0)
    assert rel(r["q_fine"], q_ref) < TOL[prec]


def test_3d_uniform_state_is_the_scalar_recurrence(mlq):
    # spatially constant v, w: K 1 = 0 and M c1 = c M1, so every node follows
    # v+ = v + dt R(v, w), w+ = w + dt eps (v - gam w); Q = |D| v
    dims = (7, 7, 4)
    mesh = O.mesh3d(*dims)
    K = 3
    phi = np.random.default_rng(0).normal(size=(mesh.ne, K))
    v, w, dt = 0.37, 0.05, 0.05
    with mlq.Context(0, 0) as ctx:
        ctx.add_level(0, dims, dt, 30)
        ctx.set_kl(0, phi)
        ctx.set_initial_state(0, np.full(mesh.n, v), np.full(mesh.n, w))
        r = ctx.solve(0, inputs.gaussian_xi(1, 0, 0, 2, K))
    a, eps, gam = 0.1, 0.01, 0.5
    for _ in range(30):
        v, w = v + dt * (v * (v - a) * (1 - v) - w), w + dt * eps * (v - gam * w)
    assert np.allclose(r["q_fine"], 0.25 * v, rtol=1e-12, atol=0)


@pytest.mark.parametrize("prec", [0, 1])
def test_3d_level_pair_and_telescoping(mlq, prec):
    # nested Kuhn levels (9,9,5) -> (5,5,3) -> (3,3,2): the coarse member of
    # a pair is the fine member of the pair below, bit for bit, and the
    # differences telescope
    dims = [(3, 3, 2), (5, 5, 3), (9, 9, 5)]
    fine = O.mesh3d(*dims[-1])
    modes, _ = O.kl_build(fine, 0.09, 0.15 ** 2, 4)
    phis = [O.centroid_table(fine, modes, O.mesh3d(*d)) for d in dims]
    dts = [0.1, 0.05, 0.025]
    xi = inputs.gaussian_xi(2, 3, 0, 4, 4)
    qref = [O.solve_batch(O.mesh3d(*d), ph, xi, dt, int(round(0.4 / dt)), v0=O.initial_state(O.mesh3d(*d), 0.3)[0],
                          nthreads=2)[0] for d, ph, dt in zip(dims, phis, dts)]
    with mlq.Context(0, prec) as ctx:
        for l, (d, dt, ph) in enumerate(zip(dims, dts, phis)):
            ctx.add_level(l, d, dt, int(round(0.4 / dt)))
            ctx.set_kl(l, ph)
            ctx.set_initial_disk(l, 0.3)
        r2 = ctx.solve(2, xi, with_coarse=True)
        r1 = ctx.solve(1, xi, with_coarse=True)
        r0 = ctx.solve(0, xi)
    assert rel(r2["q_fine"], qref[2]) < TOL[prec]
    assert rel(r2["q_coarse"], qref[1]) < TOL[prec]
    assert rel(r1["q_coarse"], qref[0]) < TOL[prec]
    assert np.array_equal(r2["q_coarse"], r1["q_fine"])
    assert np.array_equal(r1["q_coarse"], r0["q_fine"])
    assert np.allclose(r0["y"] + r1["y"] + r2["y"], r2["q_fine"], rtol=1e-14, atol=0)


def test_3d_mlqmc_estimate_matches_oracle(mlq):
    # the configuration's estimator on 3D levels: randomly shifted rank-1
    # lattice points mapped to Gaussians (one shift set per level), MLMC sums
    # over the level differences
    dims = [(5, 5, 3), (9, 9, 5)]
    fine = O.mesh3d(*dims[-1])
    K = 4
    modes, lam = O.kl_build(fine, 0.09, 0.15 ** 2, K)
    phis = [O.centroid_table(fine, modes, O.mesh3d(*d)) for d in dims]
    dts = [0.05, 0.025]
    # 8 lattice points x 2 random shifts per level, product weights lambda_k / lambda_1
    xis = [inputs.qmc_xi(0, l, 8, 2, K, lam / lam[0]).reshape(16, K) for l in range(2)]
    with mlq.Context(0, 1) as ctx:
        for l, (d, dt, ph) in enumerate(zip(dims, dts, phis)):
            ctx.add_level(l, d, dt, int(round(0.2 / dt)))
            ctx.set_kl(l, ph)
            ctx.set_initial_disk(l, 0.3)
        mean, var, rmse, ys = ctx.estimate(xis, return_y=True)
    yref = []
    for l in range(2):
        qf = O.solve_batch(O.mesh3d(*dims[l]), phis[l], xis[l], dts[l], int(round(0.2 / dts[l])),
                           v0=O.initial_state(O.mesh3d(*dims[l]), 0.3)[0], nthreads=2)[0]
        if l == 0:
            yref.append(qf)
        else:
            qc = O.solve_batch(O.mesh3d(*dims[l - 1]), phis[l - 1], xis[l], dts[l - 1], int(round(0.2 / dts[l - 1])),
                               v0=O.initial_state(O.mesh3d(*dims[l - 1]), 0.3)[0], nthreads=2)[0]
            yref.append(qf - qc)
    est_ref, _, _ = O.mlmc_estimate(yref)
    for l in range(2):
        assert np.max(np.abs(ys[l] - yref[l])) < 1e-6 * np.max(np.abs(yref[0]))
    assert abs(mean - est_ref) < 1e-6 * abs(est_ref)


# --------------------------------------------------------------------------
# Full-size 3D levels in the launch shapes of the estimate (257 x 257 x 65
# with 16 samples: clusters of 16; 129 x 129 x 33 with 64 samples: clusters
# of 4), checked by properties that hold at any size and, at 129 x 129 x 33,
# on sampled xi against the oracle over two time blocks.
# --------------------------------------------------------------------------
def lumped_mass(mesh):
    # row sums of the P1 mass matrix: |e| / 4 per vertex of every tetrahedron
    hx, hy, hz = (L / (m - 1) for L, m in zip(mesh.lengths, mesh.dims))
    return np.bincount(mesh.conn.ravel(), minlength=mesh.n) * (hx * hy * hz / 6.0 / 4.0)


def test_3d_full_size_block_conserves_mass_weighted_state(mlq):
    # K 1 = 0, so one block gives m^T v+ = 1^T (M + dt K) v+ = 1^T M y with
    # y = v + dt R(v, w): the QoI after one block is m^T y, for any fibres
    dims, dt, S = (257, 257, 65), 0.00625, 16
    mesh = O.mesh3d(*dims)
    rng = np.random.default_rng(7)
    phi = rng.normal(scale=0.5, size=(mesh.ne, 2))
    v0 = rng.uniform(0, 1, size=mesh.n)
    w0 = rng.uniform(0, 0.2, size=mesh.n)
    y = v0 + dt * (v0 * (v0 - 0.1) * (1 - v0) - w0)
    expect = lumped_mass(mesh) @ y
    with mlq.Context(0, 1) as ctx:
        ctx.add_level(0, dims, dt, 1)
        ctx.set_kl(0, phi)
        ctx.set_initial_state(0, v0, w0)
        ctx.set_profiling(True)
        r = ctx.solve(0, inputs.gaussian_xi(3, 3, 0, S, 2))
        # the launch the bench times: 16 samples, every group resident at once
        # (clusters, or > 16 CTAs per sample in one cooperative launch)
        assert ctx.member_profile()[0]["cluster"] >= 12
    assert np.all(r["status"] == 0)
    assert np.max(np.abs(r["q_fine"] - expect)) < 1e-9 * abs(expect)


def test_3d_full_size_uniform_state(mlq):
    dims, dt, S, nb = (257, 257, 65), 0.00625, 16, 12
    mesh = O.mesh3d(*dims)
    phi = np.random.default_rng(8).normal(size=(mesh.ne, 1))
    v, w = 0.45, 0.03
    with mlq.Context(0, 1) as ctx:
        ctx.add_level(0, dims, dt, nb)
        ctx.set_kl(0, phi)
        ctx.set_initial_state(0, np.full(mesh.n, v), np.full(mesh.n, w))
        r = ctx.solve(0, inputs.gaussian_xi(4, 3, 0, S, 1))
    for _ in range(nb):
        v, w = v + dt * (v * (v - 0.1) * (1 - v) - w), w + dt * 0.01 * (v - 0.5 * w)
    assert np.all(r["status"] == 0)
    assert np.allclose(r["q_fine"], 0.25 * v, rtol=1e-9, atol=0)


def test_3d_level2_sampled_against_oracle(mlq):
    dims, dt, S, nb, K = (129, 129, 33), 0.0125, 64, 2, 4
    mesh = O.mesh3d(*dims)
    modes, _ = O.kl_build(mesh, 0.09, 0.15 ** 2, K)
    phi = O.centroid_table(mesh, modes, mesh)
    xi = inputs.gaussian_xi(0, 2, 0, S, K)
    with mlq.Context(0, 1) as ctx:
        ctx.add_level(0, dims, dt, nb)
        ctx.set_kl(0, phi)
        ctx.set_profiling(True)
        r = ctx.solve(0, xi)
        assert ctx.member_profile()[0]["cluster"] == 4
    assert np.all(r["status"] == 0)
    pick = [0, 37, 63]
    v0, _ = O.initial_state(mesh, 0.1)
    q_ref, _, st = O.solve_batch(mesh, phi, xi[pick], dt, nb, v0=v0, nthreads=3)
    assert np.all(st == 0)
    assert rel(r["q_fine"][pick], q_ref) < TOL[1]
