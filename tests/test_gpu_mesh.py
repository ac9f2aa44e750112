"""Levels on general tetrahedral meshes (mlq_mesh_*): the synthetic
left-ventricle shell with wall-tangent fibre frames and helix angles, against
the FP64 oracle on the same seeded inputs (FP64 path: 1e-10 relative per
sample), plus the properties that hold at any size."""
import numpy as np
import pytest

import oracle as O
from paper_2105_02007_gb300 import inputs
from paper_2105_02007_gb300 import lv_inputs as LV

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


def test_mesh_level_matches_oracle_on_the_shell(mlq):
    xyz, conn = LV.lv_mesh(2, 8, 14)
    frames, alpha = LV.lv_fibres(xyz, conn)
    mesh = O.unstructured_mesh(xyz, conn)
    fine_xyz, fine_conn = LV.lv_mesh(3, 11, 19)           # KL on an unrelated finer shell
    modes, _ = O.kl_build(O.unstructured_mesh(fine_xyz, fine_conn), 0.09, 0.15 ** 2, 4)
    phi = O.centroid_table_unrelated(O.unstructured_mesh(fine_xyz, fine_conn), modes, mesh)
    xi = inputs.gaussian_xi(0, 0, 0, 5, 4)
    v0, w0 = LV.stimulus(xyz, radius=0.4)
    dt, nb = 0.05, 12
    q_ref, _, st = O.solve_batch(mesh, phi, xi, dt, nb, v0=v0, w0=w0, theta_mean=alpha, frames=frames, nthreads=2)
    assert np.all(st == 0)
    with mlq.MeshLevel(xyz, conn, frames) as lvl:
        lvl.set_kl(phi, alpha)
        q, status, iters = lvl.solve(xi, dt, nb, v0, w0)
    assert np.all(status == 0) and np.all(iters > 0)
    assert np.max(np.abs(q - q_ref) / np.abs(q_ref)) < 1e-10


def test_mesh_level_conservation_and_uniform_state(mlq):
    xyz, conn = LV.lv_mesh(3, 12, 20)
    frames, alpha = LV.lv_fibres(xyz, conn)
    mesh = O.unstructured_mesh(xyz, conn)
    rp, ci, mv, _ = O.assemble(mesh)
    m = np.zeros(mesh.n)
    np.add.at(m, ci, mv)
    rng = np.random.default_rng(2)
    v0, w0, dt = rng.uniform(0, 1, mesh.n), rng.uniform(0, 0.2, mesh.n), 0.02
    phi = rng.normal(scale=0.3, size=(mesh.ne, 2))
    xi = inputs.gaussian_xi(1, 0, 0, 3, 2)
    with mlq.MeshLevel(xyz, conn, frames) as lvl:
        lvl.set_kl(phi, alpha)
        q, st, _ = lvl.solve(xi, dt, 1, v0, w0)
        assert np.all(st == 0)
        assert np.allclose(q, m @ (v0 + dt * (v0 * (v0 - 0.1) * (1 - v0) - w0)), rtol=1e-11, atol=0)
        v, w = 0.4, 0.02
        q, st, _ = lvl.solve(xi, dt, 10, np.full(mesh.n, v), np.full(mesh.n, w))
    for _ in range(10):
        v, w = v + dt * (v * (v - 0.1) * (1 - v) - w), w + dt * 0.01 * (v - 0.5 * w)
    assert np.all(st == 0)
    assert np.allclose(q, m.sum() * v, rtol=1e-11, atol=0)


def test_mesh_level_rejects_bad_input(mlq):
    xyz, conn = LV.lv_mesh(1, 3, 5)
    with pytest.raises(mlq.MLQError):
        mlq.MeshLevel(xyz, np.where(conn == 1, xyz.shape[0] + 3, conn))
    flat = conn.copy()
    flat[0, 3] = flat[0, 2]                                  # degenerate tetrahedron
    with pytest.raises(mlq.MLQError):
        mlq.MeshLevel(xyz, flat)


def test_pimped_ml_over_unrelated_shells_matches_oracle(mlq):
    # eq. PimpedML over three unrelated shell meshes: term l is the QoI on
    # mesh L-l alone at the first N_l points; the library's members and
    # combination against the oracle's solves and combination (FP64 path)
    meshes = [LV.lv_mesh(*d) for d in ((2, 6, 10), (2, 8, 14), (3, 11, 19))]
    fine = O.unstructured_mesh(*meshes[-1])
    modes, _ = O.kl_build(fine, 0.09, 0.15 ** 2, 4)
    N = [2, 4, 8]
    xi = inputs.gaussian_xi(40, 0, 0, N[-1], 4)
    dt, nb = 0.05, 6
    L = len(meshes) - 1
    F_lib, F_or = [], []
    for l in range(L + 1):
        xyz, conn = meshes[L - l]
        frames, alpha = LV.lv_fibres(xyz, conn)
        mesh = O.unstructured_mesh(xyz, conn)
        phi = O.centroid_table_unrelated(fine, modes, mesh)
        v0, w0 = LV.stimulus(xyz, radius=0.4)
        q_or = O.solve_batch(mesh, phi, xi[: N[l]], dt, nb, v0=v0, w0=w0, theta_mean=alpha, frames=frames,
                             nthreads=2)[0]
        with mlq.MeshLevel(xyz, conn, frames) as lvl:
            lvl.set_kl(phi, alpha)
            q, st, _ = lvl.solve(xi[: N[l]], dt, nb, v0, w0)
        assert np.all(st == 0)
        F_lib.append(q)
        F_or.append(q_or)
    est = mlq.pimped_ml_combine(F_lib, N)
    ref = O.pimped_ml_estimate(F_or, N)
    assert abs(est - ref) <= 1e-10 * abs(ref)


@pytest.mark.parametrize("prec,cluster", [(0, 1), (0, 4), (1, 0), (1, 1), (1, 2), (1, 16), (0, 24), (1, 72)])
def test_mesh_level_precisions_and_clusters(mlq, prec, cluster):
    # the device-resident member in both precisions, on every cluster size
    # (ragged row bands) and as a cooperative launch of 24 / 72 CTAs per
    # sample (global-memory barriers and sums), against the oracle: FP64
    # 1e-10, mixed 1e-6
    xyz, conn = LV.lv_mesh(*((3, 16, 28) if cluster == 16 else (2, 8, 14)))   # 16 CTAs need >= 1024 rows
    frames, alpha = LV.lv_fibres(xyz, conn)
    mesh = O.unstructured_mesh(xyz, conn)
    modes, _ = O.kl_build(mesh, 0.09, 0.15 ** 2, 4)
    phi = O.centroid_table_unrelated(mesh, modes, mesh)
    xi = inputs.gaussian_xi(41, 0, 0, 4, 4)
    v0, w0 = LV.stimulus(xyz, radius=0.4)
    dt, nb = 0.05, 10
    q_ref, _, st = O.solve_batch(mesh, phi, xi, dt, nb, v0=v0, w0=w0, theta_mean=alpha, frames=frames, nthreads=2)
    assert np.all(st == 0)
    tol = 1e-10 if prec == 0 else 1e-6
    with mlq.MeshLevel(xyz, conn, frames) as lvl:
        lvl.set_kl(phi, alpha)
        q, status, iters = lvl.solve(xi, dt, nb, v0, w0, precision=prec, cluster=cluster)
    assert np.all(status == 0) and np.all(iters > 0)
    assert np.max(np.abs(q - q_ref) / np.abs(q_ref)) < tol


@pytest.mark.parametrize("dim", [2, 3])
def test_device_point_location_matches_host_and_oracle(mlq, dim):
    # the device transfer (bucket grid, location, the global scan of points
    # outside, interpolation) against the host helper and the oracle, on
    # unrelated shells with centroids inside and outside the located mesh,
    # and on a 2D mesh with points on shared edges and outside
    rng = np.random.default_rng(60 + dim)
    if dim == 3:
        fine_xyz, fine_conn = LV.lv_mesh(3, 11, 19)
        cx, cc = LV.lv_mesh(2, 7, 12)
        pts = cx[cc].mean(axis=1)
    else:
        m = O.mesh2d(9)
        fine_xyz, fine_conn = m.xyz, m.conn
        pts = np.vstack([rng.uniform(-0.05, 1.05, size=(200, 2)), m.xyz[::3],
                         0.5 * (m.xyz[m.conn[:40, 0]] + m.xyz[m.conn[:40, 1]])])
    f = rng.normal(size=(fine_xyz.shape[0], 5))
    dev = mlq.p1_at_points(fine_xyz, fine_conn, f, pts, device=True)
    host = mlq.p1_at_points(fine_xyz, fine_conn, f, pts)
    ref = O.p1_at_points(O.unstructured_mesh(fine_xyz, fine_conn), f, pts)
    assert np.max(np.abs(dev - host)) < 1e-12 * np.max(np.abs(host))
    assert np.max(np.abs(dev - ref)) < 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("prec", [0, 1])
def test_general_levels_in_the_context(mlq, prec):
    # unrelated shells as levels 0..2 of one context (mlq_add_level_mesh):
    # mlq_solve with the coarse member equals the standalone general-mesh
    # solver sample by sample, and mlq_estimate (eq. StandardML with MC rules,
    # Y_l = Q_l - Q_{l-1} on the same xi, each Q on its own mesh) equals the
    # oracle's solves on the three meshes: FP64 1e-10, mixed 1e-6
    meshes = [LV.lv_mesh(*d) for d in ((2, 6, 10), (2, 8, 14), (3, 11, 19))]
    fine = O.unstructured_mesh(*meshes[-1])
    modes, _ = O.kl_build(fine, 0.09, 0.15 ** 2, 4)
    N = [8, 4, 2]
    xis = [inputs.gaussian_xi(42, l, 0, N[l], 4) for l in range(3)]
    dt, nb = 0.05, 6
    tol = 1e-10 if prec == 0 else 1e-6
    lv = []
    for l, (xyz, conn) in enumerate(meshes):
        frames, alpha = LV.lv_fibres(xyz, conn)
        mesh = O.unstructured_mesh(xyz, conn)
        phi = O.centroid_table_unrelated(fine, modes, mesh)
        v0, w0 = LV.stimulus(xyz, radius=0.4)
        lv.append((xyz, conn, frames, alpha, mesh, phi, v0, w0))
    with mlq.Context(0, prec) as ctx:
        for l, (xyz, conn, frames, alpha, mesh, phi, v0, w0) in enumerate(lv):
            ctx.add_level_mesh(l, xyz, conn, dt, nb, frames=frames)
            ctx.set_kl(l, phi, alpha)
            ctx.set_initial_state(l, v0, w0)
        r = ctx.solve(2, xis[2], with_coarse=True)
        mean, var, rmse, ys = ctx.estimate(xis, return_y=True)
        # the structured-only calls refuse a general level
        with pytest.raises(mlq.MLQError) as e:
            ctx.autotune(2, xis[2])
        assert e.value.code == mlq.MLQ_EUNSUPPORTED
    assert np.all(r["status"] == 0)
    for l, key in ((2, "q_fine"), (1, "q_coarse")):
        xyz, conn, frames, alpha, mesh, phi, v0, w0 = lv[l]
        with mlq.MeshLevel(xyz, conn, frames) as m:
            m.set_kl(phi, alpha)
            q, st, _ = m.solve(xis[2], dt, nb, v0, w0, precision=prec)
        assert np.all(st == 0)
        assert np.array_equal(r[key], q), (key, r[key], q)
    assert np.array_equal(r["y"], r["q_fine"] - r["q_coarse"])
    ref_y = []
    for l in range(3):
        q_f = O.solve_batch(lv[l][4], lv[l][5], xis[l], dt, nb, v0=lv[l][6], w0=lv[l][7], theta_mean=lv[l][3],
                            frames=lv[l][2], nthreads=2)[0]
        q_c = 0.0
        if l > 0:
            q_c = O.solve_batch(lv[l - 1][4], lv[l - 1][5], xis[l], dt, nb, v0=lv[l - 1][6], w0=lv[l - 1][7],
                                theta_mean=lv[l - 1][3], frames=lv[l - 1][2], nthreads=2)[0]
        ref_y.append(q_f - q_c)
    ref = sum(float(np.mean(y)) for y in ref_y)
    scale = max(abs(float(np.mean(lv_q))) for lv_q in ref_y)
    assert abs(mean - ref) <= tol * scale
    for l in range(3):
        d = tol * scale   # bound on every per-sample error of Y_l
        assert np.max(np.abs(ys[l] - ref_y[l])) <= d
        # a sample variance moves by at most 2 sqrt(var) d + d^2 when every
        # sample moves by at most d (the unbiased estimator, N_l >= 2)
        v_ref = float(np.var(ref_y[l], ddof=1))
        assert abs(var[l] - v_ref) <= 2.0 * np.sqrt(v_ref) * d * N[l] / (N[l] - 1) + 2.0 * d * d * N[l] / (N[l] - 1)


@pytest.mark.parametrize("prec", [0, 1])
def test_state_and_synthesis_on_a_general_level(mlq, prec):
    # the field QoI (v_h(T), w(T) node by node) and the KL table (eq.
    # KLlowrank, FP64 on this solver in both precisions) of a shell level of
    # a context, against the oracle; Q of the state call equals mlq_solve's
    xyz, conn = LV.lv_mesh(2, 8, 14)
    mesh = O.unstructured_mesh(xyz, conn)
    rng = np.random.default_rng(72)
    phi = rng.normal(scale=0.3, size=(conn.shape[0], 4))
    alpha = rng.uniform(-1.0, 1.0, size=conn.shape[0])
    xi = inputs.gaussian_xi(45, 0, 0, 4, 4)
    v0, w0 = LV.stimulus(xyz, radius=0.4)
    dt, nb = 0.05, 10
    q_ref, V, W, st = O.solve_states(mesh, phi, xi, dt, nb, v0=v0, w0=w0, theta_mean=alpha)
    assert np.all(st == 0)
    with mlq.Context(0, prec) as ctx:
        ctx.add_level_mesh(0, xyz, conn, dt, nb)
        ctx.set_kl(0, phi, alpha)
        ctx.set_initial_state(0, v0, w0)
        r = ctx.solve_state(0, xi)
        plain = ctx.solve(0, xi)
        cs2 = ctx.synthesize(0, xi)
    assert np.all(r["status"] == 0)
    assert np.array_equal(r["q"], plain["q_fine"])
    tol = 1e-10 if prec == 0 else 1e-6
    assert np.max(np.abs(r["v"] - V)) <= tol * np.max(np.abs(V))
    assert np.max(np.abs(r["w"] - W)) <= tol * np.max(np.abs(W)) + tol * np.max(np.abs(V))
    assert np.max(np.abs(r["q"] - q_ref) / np.abs(q_ref)) <= tol
    assert np.max(np.abs(cs2 - O.kl_synthesis(phi, xi, alpha))) < 1e-13


@pytest.mark.parametrize("prec", [0, 1])
def test_point_qois_on_a_general_level(mlq, prec):
    # the point QoIs of Sec. 2.4 on a shell level of a context: traces
    # u(x_p, t_n) element by element against the oracle (FP64 1e-10, mixed
    # 1e-6 of max |u|) and activation times within the bound a trace error
    # gives them; the points do not change the solve
    xyz, conn = LV.lv_mesh(2, 8, 14)
    mesh = O.unstructured_mesh(xyz, conn)
    rng = np.random.default_rng(71)
    phi = rng.normal(scale=0.3, size=(conn.shape[0], 4))
    xi = inputs.gaussian_xi(44, 0, 0, 3, 4)
    v0, w0 = LV.stimulus(xyz, radius=0.4)
    # slower diffusion than the default (s_l = 0.01, s_t = 0.002) so that the
    # excitation travels over the shell within T = 30
    dt, nb, th = 0.5, 60, 0.5
    model = dict(s_l=0.01, s_t=0.002)
    # element centroids: in the stimulus, outside it at rising distance, the
    # farthest one, and a mesh node
    cen = xyz[conn].mean(axis=1)
    vc = v0[conn].mean(axis=1)
    out = np.nonzero(vc == 0)[0]
    near = out[np.argsort(np.linalg.norm(cen[out] - cen[np.argmax(vc)], axis=1))]
    pts = np.vstack([cen[np.argmax(vc)], cen[near[0]], cen[near[len(near) // 8]], cen[near[len(near) // 3]],
                     cen[near[-1]], xyz[conn[5, 2]]])
    tr, act, q, st = O.solve_points(mesh, phi, xi, dt, nb, pts, th, v0=v0, w0=w0, model=model)
    assert np.all(st == 0)
    assert np.any(act == 0) and np.any(act > 0) and np.any(act < 0)
    with mlq.Context(0, prec) as ctx:
        ctx.set_model(**model)
        ctx.add_level_mesh(0, xyz, conn, dt, nb)
        ctx.set_kl(0, phi)
        ctx.set_initial_state(0, v0, w0)
        ctx.set_points(0, pts, th)
        r = ctx.solve_points(0, xi)
        plain = ctx.solve(0, xi)
        with pytest.raises(mlq.MLQError):
            ctx.set_points(0, np.array([[9.0, 9.0, 9.0]]), th)
    assert np.all(r["status"] == 0)
    assert np.array_equal(r["q"], plain["q_fine"])
    tol = 1e-10 if prec == 0 else 1e-6
    scale = np.max(np.abs(tr))
    assert np.max(np.abs(r["trace"] - tr)) <= tol * scale
    assert np.array_equal(r["act"] < 0, act < 0) or prec == 1
    for s_, p_ in zip(*np.nonzero((act >= 0) & (r["act"] >= 0))):
        u = tr[s_, p_]
        n = max(1, int(np.ceil(act[s_, p_] / dt - 1e-9)))
        du = max(u[n] - u[n - 1], 1e-300)
        assert abs(r["act"][s_, p_] - act[s_, p_]) <= dt * 4 * tol * scale / du + 1e-12 or \
            abs(u[n] - th) <= 10 * tol * scale, (s_, p_)


def test_mesh_level_cooperative_shape_chosen_and_captured(mlq):
    # one or two samples on a ~49k-node shell: the chosen shape spreads each
    # sample over more CTAs than a cluster holds (a cooperative launch); its
    # Q agrees with clusters of 16 (another summation order) to 1e-10; in a
    # context the estimate gives the same samples eagerly and replayed from
    # a captured graph, equal to the standalone solver
    xyz, conn = LV.lv_mesh(8, 56, 98)
    frames, alpha = LV.lv_fibres(xyz, conn)
    rng = np.random.default_rng(70)
    phi = rng.normal(scale=0.3, size=(conn.shape[0], 4))
    xi = inputs.gaussian_xi(43, 0, 0, 2, 4)
    v0, w0 = LV.stimulus(xyz, radius=0.4)
    dt, nb = 0.05, 3
    with mlq.MeshLevel(xyz, conn, frames) as lvl:
        lvl.set_kl(phi, alpha)
        q_cl, st_cl, it_cl = lvl.solve(xi[:1], dt, nb, v0, w0, precision=0, cluster=16)
        q_auto, st_a, it_a = lvl.solve(xi[:1], dt, nb, v0, w0, precision=0)
        q_two, st_two, _ = lvl.solve(xi, dt, nb, v0, w0, precision=0)
    assert np.all(st_cl == 0) and np.all(st_a == 0) and np.all(st_two == 0)
    assert abs(q_auto[0] - q_cl[0]) <= 1e-10 * abs(q_cl[0])
    res = []
    for graphs in (0, 1):
        with mlq.Context(0, 0, graphs=graphs) as ctx:
            ctx.add_level_mesh(0, xyz, conn, dt, nb, frames=frames)
            ctx.set_kl(0, phi, alpha)
            ctx.set_initial_state(0, v0, w0)
            cps = ctx.level_launch(0)[0]
            for _ in range(2):   # the second call replays the captured graph
                mean, var, rmse, ys = ctx.estimate([xi], return_y=True)
            res.append(ys[0])
    assert cps > 16
    assert np.array_equal(res[0], res[1])
    assert np.array_equal(res[0], q_two)


def test_group_barrier_times_out_and_the_device_stays_usable(mlq):
    # the global-memory barrier of the cooperative shapes: exact sums over
    # many rounds; a group that counts a CTA which is never launched makes
    # the wait run out (nothing sets the flag it waits for): the call reports
    # MLQ_ETIMEOUT and the next launches and a solve work as before
    assert mlq.group_selftest(ctas=16, rounds=50) == 0
    assert mlq.group_selftest(ctas=1, rounds=3) == 0
    assert mlq.group_selftest(ctas=8, rounds=5, missing=1, max_polls=20000) == mlq.MLQ_ETIMEOUT
    assert mlq.group_selftest(ctas=16, rounds=10) == 0
    xyz, conn = LV.lv_mesh(2, 8, 14)
    frames, alpha = LV.lv_fibres(xyz, conn)
    mesh = O.unstructured_mesh(xyz, conn)
    modes, _ = O.kl_build(mesh, 0.09, 0.15 ** 2, 4)
    phi = O.centroid_table_unrelated(mesh, modes, mesh)
    v0, w0 = LV.stimulus(xyz, radius=0.4)
    xi = inputs.gaussian_xi(44, 0, 0, 2, 4)
    with mlq.MeshLevel(xyz, conn, frames) as lvl:
        lvl.set_kl(phi, alpha)
        q, st, _ = lvl.solve(xi, 0.05, 3, v0, w0, precision=0, cluster=24)
    assert np.all(st == 0) and np.all(np.isfinite(q))
