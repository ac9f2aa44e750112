"""The C ABI: the library builds, loads, exports every declared symbol, and
its host-side setup (KL builder, midpoint transfer) agrees with the oracle
through invariants (no GPU needed)."""
import os
import re

import numpy as np
import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def mlq():
    from paper_2105_02007_gb300 import build

    build.build()
    from paper_2105_02007_gb300 import mlq as m

    return m


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "mlq.h")).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(mlq_\w+)\s*\(", src, flags=re.M)))


def test_header_symbols_exported(mlq):
    syms = declared_symbols()
    assert len(syms) >= 15
    for s in syms:
        assert hasattr(mlq._lib, s), s
    assert set(syms) == set(mlq.EXPORTED)


def test_error_strings_and_bad_arguments(mlq):
    assert mlq._lib.mlq_strerror(0) == b"ok"
    assert mlq._lib.mlq_strerror(-1) == b"invalid argument"
    with pytest.raises(mlq.MLQError):
        mlq.build_kl(1, 0.09, 0.04, 4)          # m < 2
    with pytest.raises(mlq.MLQError):
        mlq.build_kl(5, 0.09, 0.04, 26)         # K > n


def test_product_kl_matches_oracle_invariants(mlq):
    m, K = 17, 10
    pm, pl = mlq.build_kl(m, 0.09, 0.04, K)
    mesh = O.mesh2d(m)
    om, ol = O.kl_build(mesh, 0.09, 0.04, K)
    assert np.allclose(pl, ol, rtol=1e-11, atol=1e-15)
    rp, ci, mv, _ = O.assemble(mesh)
    M = O.csr_to_dense(rp, ci, mv, mesh.n)
    assert np.allclose(pm.T @ M @ pm, np.diag(pl), atol=1e-13)
    # the covariance the modes represent is basis independent
    assert np.allclose(pm @ pm.T, om @ om.T, atol=1e-12)


def test_product_centroid_table_matches_oracle(mlq):
    fine = O.mesh2d(33)
    modes, _ = O.kl_build(fine, 0.09, 0.04, 5)
    for mc in (33, 17, 9, 3):
        coarse = O.mesh2d(mc)
        ref = O.centroid_table(fine, modes, coarse)
        got = mlq.centroid_table(33, modes, mc)
        assert np.allclose(got, ref, rtol=0, atol=1e-15)


def test_product_kl_3d_matches_oracle_invariants(mlq):
    # Kuhn-tetrahedra box 0.5 x 0.75 x 0.25: the same eigenvalues, M-orthogonal
    # modes and the same represented covariance as the oracle's builder
    dims, lengths, K = (6, 7, 4), (0.5, 0.75, 0.25), 8
    pm, pl = mlq.build_kl(dims, 0.09, 0.04, K, lengths=lengths)
    mesh = O.mesh3d(*dims, *lengths)
    om, ol = O.kl_build(mesh, 0.09, 0.04, K)
    assert np.allclose(pl, ol, rtol=1e-11, atol=1e-15)
    rp, ci, mv, _ = O.assemble(mesh)
    M = O.csr_to_dense(rp, ci, mv, mesh.n)
    assert np.allclose(pm.T @ M @ pm, np.diag(pl), atol=1e-13)
    assert np.allclose(pm @ pm.T, om @ om.T, atol=1e-12)


def test_product_centroid_table_3d_matches_oracle(mlq):
    fine = O.mesh3d(9, 9, 5)
    modes, _ = O.kl_build(fine, 0.09, 0.04, 4)
    for cd in ((9, 9, 5), (5, 5, 3), (3, 3, 2)):
        coarse = O.mesh3d(*cd)
        ref = O.centroid_table(fine, modes, coarse)
        got = mlq.centroid_table((9, 9, 5), modes, cd)
        assert np.allclose(got, ref, rtol=0, atol=1e-14)


@pytest.mark.parametrize("dims,ell", [((25, 25, 17), 0.15 ** 2), (97, 0.04)])
def test_product_kl_over_several_chunks_matches_oracle(mlq, dims, ell):
    # meshes of more than one 8192-node chunk of the threaded host builder:
    # pivots, B = L^T M L and the sign rule combine per-chunk results
    mesh = O.mesh3d(*dims) if isinstance(dims, tuple) else O.mesh2d(dims)
    assert mesh.n > 8192
    om, ol = O.kl_build(mesh, 0.09, ell, 8)
    pm, pl = mlq.build_kl(dims, 0.09, ell, 8)
    assert np.allclose(pl, ol, rtol=1e-12, atol=0)
    assert np.allclose(pm, om, rtol=0, atol=1e-12)


def test_product_kl_on_a_general_mesh_matches_oracle(mlq):
    # the left-ventricle shell (unstructured tetrahedra, more than one
    # 8192-node chunk): same eigenvalues and modes as the oracle's builder
    from paper_2105_02007_gb300 import lv_inputs as LV

    xyz, conn = LV.lv_mesh(3, 40, 70)
    mesh = O.unstructured_mesh(xyz, conn)
    assert mesh.n > 8192
    om, ol = O.kl_build(mesh, 0.09, 0.15 ** 2, 6)
    pm, pl = mlq.build_kl_mesh(xyz, conn, 0.09, 0.15 ** 2, 6)
    assert np.allclose(pl, ol, rtol=1e-12, atol=0)
    # the shell's rotational symmetry makes eigenvalues nearly equal, so the
    # modes within such a cluster are not unique: compare the represented
    # covariance V V^T (= L L^T of the pivoted Cholesky factor) on vectors
    r = np.random.default_rng(7).normal(size=(mesh.n, 3))
    cov_o, cov_p = om @ (om.T @ r), pm @ (pm.T @ r)
    assert np.max(np.abs(cov_p - cov_o)) < 1e-12 * np.max(np.abs(cov_o))
    # a 2D triangulation given as a general mesh: the same as the structured call
    m2 = O.mesh2d(17)
    pm2, pl2 = mlq.build_kl_mesh(m2.xyz, m2.conn, 0.09, 0.04, 5)
    sm2, sl2 = mlq.build_kl(17, 0.09, 0.04, 5)
    assert np.allclose(pl2, sl2, rtol=1e-12, atol=0) and np.allclose(pm2, sm2, rtol=0, atol=1e-12)
    with pytest.raises(mlq.MLQError):
        mlq.build_kl_mesh(xyz, np.where(conn == 0, xyz.shape[0], conn), 0.09, 0.04, 4)   # index out of range


def test_product_point_transfer_matches_oracle(mlq):
    from paper_2105_02007_gb300 import lv_inputs as LV

    fine_xyz, fine_conn = LV.lv_mesh(3, 17, 29)
    fine = O.unstructured_mesh(fine_xyz, fine_conn)
    coarse = O.unstructured_mesh(*LV.lv_mesh(2, 7, 11))
    cen = coarse.xyz[coarse.conn].mean(axis=1)
    # and points just outside: beyond the epicardium, inside the cavity,
    # above the base
    mu, _, _ = LV.prolate_coordinates(fine_xyz)
    epi = fine_xyz[np.abs(mu - LV.MU_EPI) < 1e-9][::7]
    endo = fine_xyz[np.abs(mu - LV.MU_ENDO) < 1e-9][::7]
    base = fine_xyz[np.abs(fine_xyz[:, 2]) < 1e-12][::5] + np.array([0.0, 0.0, 2e-3])
    pts = np.concatenate([cen, epi * 1.002, endo * 0.998, base])
    f = np.random.default_rng(6).normal(size=(fine.n, 3))
    ref, el, lam_min = O.p1_at_points(fine, f, pts, return_location=True)
    got = mlq.p1_at_points(fine_xyz, fine_conn, f, pts)
    inside = lam_min >= -1e-12
    assert (~inside).sum() > 20             # the case of points outside is exercised
    # points inside: the P1 function is continuous, any containing simplex agrees
    assert np.max(np.abs(got[inside] - ref[inside])) < 1e-12
    # points outside: the same simplex by the same rule (up to rounding of the
    # barycentric coordinates)
    assert np.max(np.abs(got[~inside] - ref[~inside])) < 1e-9


def test_mlmc_allocation_is_the_constrained_optimum(mlq):
    # closed form: V_l = 4^-l, C_l = 4^l gives N_l = (L + 1) 4^-l / eps^2
    L, eps = 4, 1e-3
    V = 4.0 ** -np.arange(L + 1)
    C = 4.0 ** np.arange(L + 1)
    N = mlq.mlmc_allocation(V, C, eps, nmin=1)
    assert np.array_equal(N, np.ceil((L + 1) * 4.0 ** -np.arange(L + 1) / eps ** 2).astype(np.int64))
    # generic: the error target holds, and no other allocation meeting it is
    # cheaper (first-order optimality: perturbations along the constraint)
    rng = np.random.default_rng(8)
    V, C, eps = rng.uniform(1e-6, 1e-3, 5), rng.uniform(1, 1e4, 5), 2e-4
    N = mlq.mlmc_allocation(V, C, eps, nmin=1)
    assert np.sum(V / N) <= eps ** 2 * (1 + 1e-12)
    n_star = np.sqrt(V / C) * np.sum(np.sqrt(V * C)) / eps ** 2
    assert np.allclose(np.sum(V / n_star), eps ** 2, rtol=1e-12)
    cost = np.sum(n_star * C)
    for _ in range(50):
        d = rng.normal(size=5) * 0.05 * n_star
        d -= (np.sum(V / n_star ** 2 * d) / np.sum((V / n_star ** 2) ** 2)) * V / n_star ** 2   # stay on the constraint to first order
        m = n_star + d
        scale = np.sum(V / m) / eps ** 2                     # restore the constraint exactly
        assert np.sum(m * scale * C) >= cost * (1 - 1e-12)
    # nmin and a level without variance
    N = mlq.mlmc_allocation([0.0, 1e-4], [1.0, 10.0], 1e-3, nmin=3)
    assert N[0] == 3 and N[1] == np.ceil(np.sqrt(1e-5) * np.sqrt(1e-3) / 1e-6)
    for bad in (dict(var=[-1.0], cost=[1.0]), dict(var=[1.0], cost=[0.0])):
        with pytest.raises(mlq.MLQError):
            mlq.mlmc_allocation(bad["var"], bad["cost"], 1e-3)


def test_trace_helpers_match_oracle(mlq):
    # time QoIs: the library's L2/H1(0,T) norms against the oracle's
    # quadrature, and the time prolongation keeps the coarse values and is
    # exact on linear functions
    rng = np.random.default_rng(9)
    e = rng.normal(size=41)
    for T in (1.0, 10.0):
        a = mlq.time_norms(e, T)
        b = O.time_norms(e, T)
        assert abs(a[0] - b[0]) <= 1e-13 * b[0] and abs(a[1] - b[1]) <= 1e-13 * b[1]
    uc = rng.normal(size=11)
    uf = mlq.trace_prolong(uc)
    assert uf.size == 21 and np.array_equal(uf[::2], uc)
    lin = 0.25 + 0.5 * np.arange(11.0)
    assert np.allclose(mlq.trace_prolong(lin), 0.25 + 0.25 * np.arange(21.0), rtol=0, atol=1e-15)
    # the prolonged coarse trace minus itself is zero in H1 (the level
    # difference of a constant-in-level trace)
    assert mlq.time_norms(mlq.trace_prolong(uc) - np.interp(np.arange(21) / 2.0, np.arange(11.0), uc), 1.0)[1] < 1e-14


@pytest.mark.parametrize("m", [(5,), (9,), (5, 4, 3), (3, 5, 3)])
def test_field_prolong_is_the_p1_interpolant(mlq, m):
    # the library's transfer against the oracle's point location on the
    # coarse mesh, evaluated at the fine nodes (exact for nested P1)
    rng = np.random.default_rng(len(m) * 10 + m[0])
    if len(m) == 1:
        coarse, fine = O.mesh2d(m[0]), O.mesh2d(2 * m[0] - 1)
        arg = m[0]
    else:
        coarse = O.mesh3d(*m)
        fine = O.mesh3d(*[2 * v - 1 for v in m])
        arg = m
    vc = rng.normal(size=coarse.n)
    vf = mlq.field_prolong(arg, vc)
    ref = O.p1_at_points(coarse, vc[:, None], fine.xyz)[:, 0]
    assert np.max(np.abs(vf - ref)) < 1e-14
    # linear fields are reproduced exactly
    lin = coarse.xyz @ np.arange(1.0, coarse.dim + 1.0) + 0.5
    assert np.max(np.abs(mlq.field_prolong(arg, lin) - (fine.xyz @ np.arange(1.0, coarse.dim + 1.0) + 0.5))) < 1e-13


@pytest.mark.parametrize("m", [9, (5, 4, 3)])
def test_field_norms_match_assembled_matrices(mlq, m):
    mesh = O.mesh2d(m) if np.ndim(m) == 0 else O.mesh3d(*m)
    rng = np.random.default_rng(3)
    e = rng.normal(size=mesh.n)
    rp, ci, mv, kv = O.assemble(mesh, None, 1.0, 1.0)      # isotropic: the H1 seminorm's matrix
    M = O.csr_to_dense(rp, ci, mv, mesh.n)
    K = O.csr_to_dense(rp, ci, kv, mesh.n)
    l2, h1 = mlq.field_norms(m, e)
    assert abs(l2 ** 2 - e @ M @ e) <= 1e-12 * (e @ M @ e)
    assert abs(h1 ** 2 - e @ (M + K) @ e) <= 1e-12 * (e @ (M + K) @ e)


def test_pimped_ml_combine_matches_oracle(mlq):
    rng = np.random.default_rng(12)
    N = [3, 9, 27, 40]
    F = [rng.normal(1.0 + l, 0.1, N[l]) for l in range(4)]
    assert abs(mlq.pimped_ml_combine(F, N) - O.pimped_ml_estimate(F, N)) < 1e-14
    with pytest.raises(mlq.MLQError):
        mlq.pimped_ml_combine(F, [3, 2, 27, 40])            # rules must be nested
