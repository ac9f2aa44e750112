"""Pins of the oracle's parts for non-nested levels on the synthetic
left-ventricle shell (CPU): the mesh generator, the fibre frames, the
frame-aware assembly, P1 point location between unrelated meshes and the
estimator of eq. PimpedML.  Each pin checks against something other than the
code under test: exact volumes, orthogonality, the x-y special case pinned
elsewhere, invariance under rotation, exactness on linear fields, the
conservation identity and the algebraic identity with eq. StandardML.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2105_02007_gb300 import inputs
from paper_2105_02007_gb300 import lv_inputs as LV


def tet_volumes(xyz, conn):
    X = xyz[conn]
    return np.einsum("ij,ij->i", np.cross(X[:, 1] - X[:, 0], X[:, 2] - X[:, 0]), X[:, 3] - X[:, 0]) / 6.0


@pytest.mark.parametrize("res", [(1, 3, 5), (2, 6, 8), (4, 40, 100)])
def test_lv_mesh_conforming_closed_oriented(res):
    xyz, conn = LV.lv_mesh(*res)
    n_mu, n_nu, n_phi = res
    assert xyz.shape[0] == (n_mu + 1) * (n_nu * n_phi + 1)
    assert conn.shape[0] == 6 * n_mu * (n_nu - 1) * n_phi + 3 * n_mu * n_phi
    assert np.all(tet_volumes(xyz, conn) > 0)
    faces = np.sort(np.concatenate([conn[:, [0, 1, 2]], conn[:, [0, 1, 3]], conn[:, [0, 2, 3]], conn[:, [1, 2, 3]]]),
                    axis=1)
    uniq, count = np.unique(faces, axis=0, return_counts=True)
    assert count.max() == 2
    # every face seen once lies on the endocardium, the epicardium or the base:
    # no crack at the seam phi = 0 or at the apex
    mu, _, _ = LV.prolate_coordinates(xyz)
    bf = uniq[count == 1]
    on = (np.abs(mu[bf] - LV.MU_ENDO) < 1e-9).all(1) | (np.abs(mu[bf] - LV.MU_EPI) < 1e-9).all(1) \
        | (np.abs(xyz[bf][:, :, 2]) < 1e-12).all(1)
    assert on.all()
    # boundary faces: endo and epi rings (two triangles per quad, the apex
    # closes with one triangle per phi cell), base quads
    assert bf.shape[0] == 2 * (2 * (n_nu - 1) * n_phi + n_phi) + 2 * n_mu * n_phi


def test_lv_mesh_volume_converges_to_the_shell():
    exact = LV.shell_volume()
    errs = [abs(tet_volumes(*LV.lv_mesh(*r)).sum() / exact - 1.0) for r in [(2, 10, 25), (4, 40, 100)]]
    assert errs[1] < 2e-3
    assert errs[1] < errs[0] / 4


def test_lv_fibre_frames():
    xyz, conn = LV.lv_mesh(4, 40, 100)
    frames, alpha = LV.lv_fibres(xyz, conn)
    e_c, e_l = frames[:, :3], frames[:, 3:]
    assert np.allclose(np.linalg.norm(e_c, axis=1), 1.0, atol=1e-14)
    assert np.allclose(np.linalg.norm(e_l, axis=1), 1.0, atol=1e-14)
    assert np.allclose(np.einsum("ij,ij->i", e_c, e_l), 0.0, atol=1e-14)
    # both tangent to the wall: orthogonal to grad mu (finite differences of mu)
    cen = xyz[conn].mean(axis=1)
    h = 1e-6
    g = np.stack([(LV.prolate_coordinates(cen + h * np.eye(3)[a])[0] - LV.prolate_coordinates(cen - h * np.eye(3)[a])[0])
                  / (2 * h) for a in range(3)], axis=1)
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    assert np.max(np.abs(np.einsum("ij,ij->i", g, e_c))) < 1e-6
    assert np.max(np.abs(np.einsum("ij,ij->i", g, e_l))) < 1e-6
    # helix angle: +60 deg at the endocardium falling linearly to -60 deg
    mu = LV.prolate_coordinates(cen)[0]
    t = (mu - LV.MU_ENDO) / (LV.MU_EPI - LV.MU_ENDO)
    assert np.allclose(alpha, np.deg2rad(60.0 - 120.0 * np.clip(t, 0, 1)), atol=1e-12)
    assert alpha.max() <= math.radians(60.0) + 1e-12 and alpha.min() >= math.radians(-60.0) - 1e-12


def test_frames_of_the_xy_axes_reduce_to_the_plane_fibres():
    mesh = O.mesh3d(6, 5, 4)
    theta = np.random.default_rng(0).normal(size=mesh.ne)
    frames = np.tile([1.0, 0.0, 0.0, 0.0, 1.0, 0.0], (mesh.ne, 1))
    a = O.assemble(mesh, theta)
    b = O.assemble(mesh, theta, frames=frames)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_frames_rotation_invariance():
    # rotating the mesh and its fibre frames together leaves M and K unchanged
    xyz, conn = LV.lv_mesh(2, 6, 8)
    frames, alpha = LV.lv_fibres(xyz, conn)
    theta = alpha + np.random.default_rng(1).normal(scale=0.3, size=conn.shape[0])
    q, _ = np.linalg.qr(np.random.default_rng(2).normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    m0 = O.unstructured_mesh(xyz, conn)
    m1 = O.unstructured_mesh(xyz @ q.T, conn)
    fr1 = np.concatenate([frames[:, :3] @ q.T, frames[:, 3:] @ q.T], axis=1)
    rp0, ci0, mv0, kv0 = O.assemble(m0, theta, frames=frames)
    rp1, ci1, mv1, kv1 = O.assemble(m1, theta, frames=fr1)
    assert np.array_equal(rp0, rp1) and np.array_equal(ci0, ci1)
    assert np.max(np.abs(mv1 - mv0)) < 1e-13 * np.max(np.abs(mv0))
    assert np.max(np.abs(kv1 - kv0)) < 1e-12 * np.max(np.abs(kv0))
    # and the fibre matters: turning the frames by 90 degrees changes K
    fr_sw = np.concatenate([frames[:, 3:], -frames[:, :3]], axis=1)
    kv_sw = O.assemble(m0, theta, frames=fr_sw)[3]
    assert np.max(np.abs(kv_sw - kv0)) > 1e-3 * np.max(np.abs(kv0))


def test_one_block_conserves_mass_weighted_state_with_frames():
    # K 1 = 0 for any fibres, so one block gives m^T v+ = m^T (v + dt R)
    xyz, conn = LV.lv_mesh(2, 8, 12)
    mesh = O.unstructured_mesh(xyz, conn)
    frames, alpha = LV.lv_fibres(xyz, conn)
    rp, ci, mv, kv = O.assemble(mesh, alpha, frames=frames)
    n = mesh.n
    ones = np.ones(n)
    K1 = np.zeros(n)
    np.add.at(K1, np.repeat(np.arange(n), np.diff(rp)), kv)
    assert np.max(np.abs(K1)) < 1e-12 * np.max(np.abs(kv))
    m = np.zeros(n)
    np.add.at(m, ci, mv)
    rng = np.random.default_rng(3)
    v0, w0, dt = rng.uniform(0, 1, n), rng.uniform(0, 0.2, n), 0.01
    phi = rng.normal(scale=0.2, size=(mesh.ne, 3))
    xi = inputs.gaussian_xi(0, 0, 0, 2, 3)
    q, _, st = O.solve_batch(mesh, phi, xi, dt, 1, v0=v0, w0=w0, theta_mean=alpha, frames=frames, nthreads=2)
    assert np.all(st == 0)
    expect = m @ (v0 + dt * (v0 * (v0 - 0.1) * (1 - v0) - w0))
    assert np.allclose(q, expect, rtol=1e-11, atol=0)


def test_p1_at_points_exact_on_linear_fields_between_unrelated_meshes():
    fine = O.unstructured_mesh(*LV.lv_mesh(3, 17, 29))
    coarse = O.unstructured_mesh(*LV.lv_mesh(2, 7, 11))
    A = np.array([[0.3, -1.2, 0.7], [2.0, 0.5, -0.4]])
    c0 = np.array([0.1, -0.3])
    f = fine.xyz @ A.T + c0
    cen = coarse.xyz[coarse.conn].mean(axis=1)
    got, el, lam_min = O.p1_at_points(fine, f, cen, return_location=True)
    assert np.all(el >= 0)
    # inside or outside the fine mesh, a P1 function reproduces a linear one
    assert np.max(np.abs(got - (cen @ A.T + c0))) < 1e-12
    inside = lam_min >= -1e-12
    assert inside.mean() > 0.8        # most centroids lie inside; the rest near the curved walls
    # the simplex reported for a point inside contains it (barycentric
    # coordinates recomputed here with a dense solve)
    idx = np.flatnonzero(inside)
    X = fine.xyz[fine.conn[el[idx]]]                       # (m, 4, 3)
    T = np.transpose(X[:, 1:] - X[:, :1], (0, 2, 1))       # columns X_a - X_0
    lam = np.linalg.solve(T, (cen[idx] - X[:, 0])[:, :, None])[:, :, 0]
    lam = np.concatenate([1.0 - lam.sum(axis=1, keepdims=True), lam], axis=1)
    assert lam.min() > -1e-10
    # nodes of the fine mesh are reproduced exactly (any simplex sharing the node)
    g = np.random.default_rng(4).normal(size=(fine.n, 2))
    assert np.max(np.abs(O.p1_at_points(fine, g, fine.xyz[::37]) - g[::37])) < 1e-12


def test_pimped_ml_identities():
    rng = np.random.default_rng(5)
    L, N = 3, [4, 9, 20, 50]
    # F_j at the first N_{L-j} points of the nested rules, one table per mesh j
    f = [rng.normal(size=N[L]) + 0.1 * j for j in range(L + 1)]
    terms = [f[L - l][:N[l]] for l in range(L + 1)]
    est = O.pimped_ml_estimate(terms, N)
    # eq. StandardML on the same rules: sum_j Q_{L-j}(F_j - F_{j-1})
    std = sum(np.mean(f[j][:N[L - j]] - (f[j - 1][:N[L - j]] if j > 0 else 0.0)) for j in range(L + 1))
    assert abs(est - std) < 1e-14 * max(1.0, abs(std))
    # one function on every mesh: the rules telescope to the finest rule
    g = rng.normal(size=N[L])
    assert abs(O.pimped_ml_estimate([g[:N[l]] for l in range(L + 1)], N) - np.mean(g)) < 1e-15


def test_non_nested_pipeline_small():
    # two unrelated LV meshes: KL on the finer one, transfer by point location,
    # per-level solves, eq. PimpedML
    meshes = [LV.lv_mesh(2, 6, 10), LV.lv_mesh(3, 9, 14)]
    fine = O.unstructured_mesh(*meshes[-1])
    modes, lam = O.kl_build(fine, 0.09, 0.15 ** 2, 4)
    assert np.all(np.diff(lam) <= 0)
    F, N = [], [3, 6]
    for l in range(2):
        mesh = O.unstructured_mesh(*meshes[1 - l])            # term l uses mesh L - l
        frames, alpha = LV.lv_fibres(mesh.xyz, mesh.conn)
        phi = O.centroid_table_unrelated(fine, modes, mesh)
        xi = inputs.gaussian_xi(0, l, 0, N[l], 4)
        v0, w0 = LV.stimulus(mesh.xyz, radius=0.4)
        assert v0.sum() > 0
        q, _, st = O.solve_batch(mesh, phi, xi, 0.05, 4, v0=v0, w0=w0, theta_mean=alpha, frames=frames,
                                 nthreads=2)
        assert np.all(st == 0) and np.all(np.isfinite(q))
        F.append(q)
    est = O.pimped_ml_estimate(F, N)
    assert np.isfinite(est) and est > 0
