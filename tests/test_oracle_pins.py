"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each check is chosen so that a plausible slip in the oracle (a dropped term,
a wrong sign or index, a transposed operand) fails at least one of them:

* mesh volumes and the mass-matrix total (Sec. 3.1);
* closed-form interior stencils: textbook 5-point / 7-point Laplacians and a
  hand-derived constant-fibre stencil (Sec. 3.1 with eq. AdmV);
* Lemma 2.1 (eigenvalues of G are g and |V|) read off the assembled matrix;
* KL: M-orthogonality and the eigenvalue identities of eqs. approxEig/redEig,
  and agreement with a dense generalised eigen-solver at full rank;
* midpoint-rule transfer (Sec. 4) exact on linear fields;
* the time-block solve against dense LU, the exact scalar recurrence for
  spatially uniform states, per-block conservation, mirror symmetry;
* the multilevel telescoping identity (eq. StandardML).
"""
import numpy as np
import pytest
import scipy.linalg

import oracle as O
from paper_2105_02007_gb300 import inputs

SL, ST = 1.0, 0.2


def simplex_volumes(mesh):
    X = mesh.xyz[mesh.conn]                      # (ne, d+1, d)
    J = X[:, 1:, :] - X[:, :1, :]
    d = mesh.dim
    return np.linalg.det(J) / (2.0 if d == 2 else 6.0)


# --------------------------------------------------------------------------
# meshes and matrices
# --------------------------------------------------------------------------
@pytest.mark.parametrize("m", [2, 5, 17])
def test_mesh2d_counts_orientation_area(m):
    mesh = O.mesh2d(m)
    assert mesh.n == m * m and mesh.ne == 2 * (m - 1) ** 2
    vol = simplex_volumes(mesh)
    assert np.all(vol > 0)                       # counter-clockwise, non-degenerate
    assert abs(vol.sum() - 1.0) < 1e-14


def test_mesh3d_counts_volume():
    mesh = O.mesh3d(4, 5, 3, 1.0, 1.0, 0.25)
    assert mesh.n == 60 and mesh.ne == 6 * 3 * 4 * 2
    vol = np.abs(simplex_volumes(mesh))
    assert np.all(vol > 0)
    assert abs(vol.sum() - 0.25) < 1e-14
    # every tetrahedron of a cube has the same volume h^3/6
    assert np.allclose(vol, vol[0], rtol=1e-13)


@pytest.mark.parametrize("mesh_fn,area", [(lambda: O.mesh2d(9), 1.0),
                                          (lambda: O.mesh3d(5, 5, 3, 1.0, 1.0, 0.25), 0.25)])
def test_mass_total_and_stiffness_kernel(mesh_fn, area):
    mesh = mesh_fn()
    rng = np.random.default_rng(1)
    rp, ci, mv, kv = O.assemble(mesh, rng.normal(size=mesh.ne), SL, ST)
    M = O.csr_to_dense(rp, ci, mv, mesh.n)
    K = O.csr_to_dense(rp, ci, kv, mesh.n)
    assert abs(M.sum() - area) < 1e-15 * 10
    assert np.max(np.abs(K.sum(axis=1))) < 1e-13          # K 1 = 0
    assert np.max(np.abs(K - K.T)) < 1e-14                # symmetric
    assert np.linalg.eigvalsh(K).min() > -1e-12           # positive semi-definite
    assert np.linalg.eigvalsh(M).min() > 0                # mass SPD


def test_mass_interior_stencil_2d():
    m = 9
    h = 1.0 / (m - 1)
    mesh = O.mesh2d(m)
    rp, ci, mv, _ = O.assemble(mesh)
    M = O.csr_to_dense(rp, ci, mv, mesh.n)
    i = 4 + m * 4
    assert abs(M[i, i] - h * h / 2) < 1e-16
    for off in (1, -1, m, -m, m + 1, -m - 1):
        assert abs(M[i, i + off] - h * h / 12) < 1e-17
    assert np.count_nonzero(M[i]) == 7


def test_isotropic_stiffness_is_textbook_laplacian():
    m = 7
    mesh = O.mesh2d(m)
    rp, ci, _, kv = O.assemble(mesh, None, 1.0, 1.0)
    K = O.csr_to_dense(rp, ci, kv, mesh.n)
    i = 3 + m * 3
    expect = {0: 4.0, 1: -1.0, -1: -1.0, m: -1.0, -m: -1.0}
    for j in range(mesh.n):
        assert abs(K[i, j] - expect.get(j - i, 0.0)) < 1e-14
    # 3D Kuhn tetrahedra: the 7-point Laplacian scaled by h
    m3 = 5
    h = 1.0 / (m3 - 1)
    mesh3 = O.mesh3d(m3, m3, m3, 1.0, 1.0, 1.0)
    rp, ci, _, kv = O.assemble(mesh3, None, 1.0, 1.0)
    K3 = O.csr_to_dense(rp, ci, kv, mesh3.n)
    i = 2 + m3 * (2 + m3 * 2)
    exp3 = {0: 6 * h, 1: -h, -1: -h, m3: -h, -m3: -h, m3 * m3: -h, -m3 * m3: -h}
    for j in range(mesh3.n):
        assert abs(K3[i, j] - exp3.get(j - i, 0.0)) < 1e-14


@pytest.mark.parametrize("th", [0.0, np.pi / 2, 0.3, -1.1])
def test_constant_fibre_stencil_closed_form(th):
    # For constant D = [[d11,d12],[d12,d22]] the P1 stencil of this
    # triangulation (derived by hand from the six triangles around a node):
    # centre 2(d11+d22-d12), E/W -(d11-d12), N/S -(d22-d12), NE/SW -d12.
    m = 7
    mesh = O.mesh2d(m)
    rp, ci, _, kv = O.assemble(mesh, np.full(mesh.ne, th), SL, ST)
    K = O.csr_to_dense(rp, ci, kv, mesh.n)
    c, s = np.cos(th), np.sin(th)
    d11 = ST + (SL - ST) * c * c
    d22 = ST + (SL - ST) * s * s
    d12 = (SL - ST) * c * s
    i = 3 + m * 3
    expect = {0: 2 * (d11 + d22 - d12), 1: -(d11 - d12), -1: -(d11 - d12), m: -(d22 - d12),
              -m: -(d22 - d12), m + 1: -d12, -m - 1: -d12}
    for j in range(mesh.n):
        assert abs(K[i, j] - expect.get(j - i, 0.0)) < 1e-14


@pytest.mark.parametrize("th", [0.0, 0.7, -2.0])
def test_lemma_2_1_eigenvalues_of_conductivity(th):
    # Lemma 2.1: G f = |V| f and G f_perp = g f_perp.  For constant D the P1
    # stiffness applied to u = (a.x)^2/2 at an interior node equals
    # -(a^T D a) times that node's lumped mass h^2, so a = f gives s_l and
    # a = f_perp gives s_t.
    m = 9
    h = 1.0 / (m - 1)
    mesh = O.mesh2d(m)
    rp, ci, _, kv = O.assemble(mesh, np.full(mesh.ne, th), SL, ST)
    K = O.csr_to_dense(rp, ci, kv, mesh.n)
    i = 4 + m * 4
    f = np.array([np.cos(th), np.sin(th)])
    fp = np.array([-np.sin(th), np.cos(th)])
    for a, lam in ((f, SL), (fp, ST)):
        u = 0.5 * (mesh.xyz @ a) ** 2
        assert abs((K @ u)[i] + lam * h * h) < 1e-13


def _lemma_2_1_check_3d(mesh, h, th, frames, dirs):
    # For constant D the P1 stiffness of a translation-invariant mesh applied
    # to u = (a.x)^2/2 at an interior node equals -(a^T D a) times the node's
    # lumped mass (h^3 on the Kuhn cube mesh): div(D grad u) = a^T D a, and the
    # stencil annihilates constants and linear fields.  With f the fibre, a = f
    # gives s_l (Lemma 2.1: G f = |V| f) and every a orthogonal to f gives s_t.
    rp, ci, _, kv = O.assemble(mesh, np.full(mesh.ne, th), SL, ST, frames=frames)
    K = O.csr_to_dense(rp, ci, kv, mesh.n)
    m = mesh.dims[0]
    interior = [i + m * (j + m * k) for i in (2, 3, 4) for j in (2, 4) for k in (3, 4)]
    for a, lam in dirs:
        u = 0.5 * (mesh.xyz @ a) ** 2
        Ku = K @ u
        for i in interior:
            assert abs(Ku[i] + lam * h ** 3) < 1e-13, (a, i, Ku[i], -lam * h ** 3)


@pytest.mark.parametrize("th", [0.0, 0.7, -2.0, 1.3])
def test_lemma_2_1_eigenvalues_of_conductivity_3d(th):
    # Kuhn tetrahedra of the unit cube, 7 x 7 x 7 nodes, in-plane fibre
    # f = (cos t, sin t, 0): f gives s_l; the in-plane normal of f and e_z give s_t.
    m = 7
    h = 1.0 / (m - 1)
    mesh = O.mesh3d(m, m, m, 1.0, 1.0, 1.0)
    f = np.array([np.cos(th), np.sin(th), 0.0])
    fp = np.array([-np.sin(th), np.cos(th), 0.0])
    ez = np.array([0.0, 0.0, 1.0])
    b = (f + ez) / np.sqrt(2.0)          # mixes both eigenvalues: s_t + (s_l - s_t)/2
    _lemma_2_1_check_3d(mesh, h, th, None, [(f, SL), (fp, ST), (ez, ST), (b, 0.5 * (SL + ST))])


@pytest.mark.parametrize("th", [0.0, 0.9, -2.4])
def test_lemma_2_1_with_frame_out_of_plane(th):
    # The fibre turns in the plane of a frame (e1, e2) tilted out of the x-y
    # plane (the ventricle's wall-tangent frames): f = cos t e1 + sin t e2
    # gives s_l, the in-frame normal -sin t e1 + cos t e2 and e1 x e2 give s_t.
    m = 7
    h = 1.0 / (m - 1)
    mesh = O.mesh3d(m, m, m, 1.0, 1.0, 1.0)
    rng = np.random.default_rng(11)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    e1, e2 = Q[:, 0], Q[:, 1]
    assert abs(e1[2]) > 0.1 and abs(e2[2]) > 0.1        # genuinely out of the x-y plane
    frames = np.tile(np.concatenate([e1, e2]), (mesh.ne, 1))
    f = np.cos(th) * e1 + np.sin(th) * e2
    fp = -np.sin(th) * e1 + np.cos(th) * e2
    nrm = np.cross(e1, e2)
    _lemma_2_1_check_3d(mesh, h, th, frames, [(f, SL), (fp, ST), (nrm, ST)])


# --------------------------------------------------------------------------
# KL expansion
# --------------------------------------------------------------------------
def _dense_cov(mesh, sigma2, ell):
    d2 = ((mesh.xyz[:, None, :] - mesh.xyz[None, :, :]) ** 2).sum(-1)
    return sigma2 * np.exp(-d2 / ell)


def test_kl_m_orthogonality_and_trace():
    mesh = O.mesh2d(17)
    K = 12
    modes, lam, L, piv = O.kl_build(mesh, 0.09, 0.04, K, return_factor=True)
    rp, ci, mv, _ = O.assemble(mesh)
    M = O.csr_to_dense(rp, ci, mv, mesh.n)
    G = modes.T @ M @ modes
    assert np.allclose(G, np.diag(lam), atol=1e-14 * lam.max() * 50)
    assert np.all(np.diff(lam) <= 0) and lam[-1] > 0
    assert abs(lam.sum() - np.trace(L.T @ M @ L)) < 1e-13
    # pivoted Cholesky reproduces C at the pivots and never overshoots it
    C = _dense_cov(mesh, 0.09, 0.04)
    R = C - L @ L.T
    assert np.max(np.abs(R[np.ix_(piv, piv)])) < 1e-12
    assert np.linalg.eigvalsh(R).min() > -1e-12
    # first pivot: all diagonals equal, tie broken towards node 0
    assert piv[0] == 0
    # truncated eigenvalue sum grows with K, bounded by tr(C M)
    trCM = float(np.sum(C * M))
    prev = 0.0
    for k in (2, 6, 12, 24):
        s = O.kl_build(mesh, 0.09, 0.04, k)[1].sum()
        assert prev < s <= trCM * (1 + 1e-12)
        prev = s
    # KL modes solve M C_K M v = lambda M v with C_K = L L^T (eq. approxEig)
    CK = L @ L.T
    for k in range(K):
        res = M @ CK @ M @ modes[:, k] - lam[k] * M @ modes[:, k]
        assert np.linalg.norm(res) < 1e-12 * np.linalg.norm(lam[k] * M @ modes[:, k]) * 1e3


def test_kl_full_rank_matches_dense_generalised_eigensolver():
    mesh = O.mesh2d(4)
    n = mesh.n
    modes, lam = O.kl_build(mesh, 0.09, 0.5, n)
    rp, ci, mv, _ = O.assemble(mesh)
    M = O.csr_to_dense(rp, ci, mv, n)
    C = _dense_cov(mesh, 0.09, 0.5)
    ref = scipy.linalg.eigh(M @ C @ M, M, eigvals_only=True)[::-1]
    big = ref > 1e-9 * ref[0]
    assert np.allclose(lam[big], ref[big], rtol=1e-8)


def test_kl_sign_convention():
    mesh = O.mesh2d(9)
    modes, _ = O.kl_build(mesh, 0.09, 0.04, 6)
    for k in range(6):
        j = int(np.argmax(np.abs(modes[:, k])))
        assert modes[j, k] > 0


def test_kl_synthesis_covariance_matches_modes():
    # The synthesised field theta = V xi with xi ~ N(0, I) has covariance
    # V V^T (the truncated KL covariance): checked on the sample covariance of
    # 20000 draws, within Monte Carlo error, through cos 2t / sin 2t moments:
    # E[cos 2t] = exp(-2 var t) for a centred Gaussian t.
    mesh = O.mesh2d(9)
    modes, _ = O.kl_build(mesh, 0.09, 0.04, 6)
    phi = O.centroid_table(mesh, modes, mesh)
    xi = inputs.gaussian_xi(11, 0, 0, 20000, 6)
    cs = O.kl_synthesis(phi, xi)
    var = np.sum(phi * phi, axis=1)
    assert np.max(np.abs(cs[:, :, 0].mean(axis=0) - np.exp(-2 * var))) < 0.02
    assert np.max(np.abs(cs[:, :, 1].mean(axis=0))) < 0.02
    theta = np.arctan2(cs[:, :, 1], cs[:, :, 0]) / 2          # |theta| < pi/2 w.h.p. here
    emp = np.cov(theta[:, :12].T)
    assert np.max(np.abs(emp - phi[:12] @ phi[:12].T)) < 0.01


# --------------------------------------------------------------------------
# midpoint-rule transfer
# --------------------------------------------------------------------------
def test_centroid_table_finest_is_vertex_mean():
    mesh = O.mesh2d(9)
    rng = np.random.default_rng(3)
    f = rng.normal(size=(mesh.n, 3))
    phi = O.centroid_table(mesh, f, mesh)
    assert np.allclose(phi, f[mesh.conn].mean(axis=1), atol=1e-14)


def test_centroid_table_exact_on_linear_fields():
    fine = O.mesh2d(17)
    coarse = O.mesh2d(5)
    f = np.stack([1.0 + 0 * fine.xyz[:, 0], fine.xyz[:, 0], 2 * fine.xyz[:, 1] - fine.xyz[:, 0]], axis=1)
    phi = O.centroid_table(fine, f, coarse)
    cen = coarse.xyz[coarse.conn].mean(axis=1)
    ref = np.stack([np.ones(coarse.ne), cen[:, 0], 2 * cen[:, 1] - cen[:, 0]], axis=1)
    assert np.allclose(phi, ref, atol=1e-14)
    fine3 = O.mesh3d(9, 9, 5)
    coarse3 = O.mesh3d(5, 5, 3)
    f3 = np.stack([fine3.xyz[:, 0] - 3 * fine3.xyz[:, 2], fine3.xyz[:, 1]], axis=1)
    phi3 = O.centroid_table(fine3, f3, coarse3)
    c3 = coarse3.xyz[coarse3.conn].mean(axis=1)
    assert np.allclose(phi3, np.stack([c3[:, 0] - 3 * c3[:, 2], c3[:, 1]], axis=1), atol=1e-14)


def test_centroid_of_nested_coarse_triangle_is_central_fine_child():
    # In red refinement the coarse centroid is the centroid of the central
    # child, so the transfer equals the fine element's own midpoint value.
    fine = O.mesh2d(9)
    coarse = O.mesh2d(5)
    rng = np.random.default_rng(5)
    f = rng.normal(size=(fine.n, 1))
    phi_c = O.centroid_table(fine, f, coarse)[:, 0]
    phi_f = O.centroid_table(fine, f, fine)[:, 0]
    cen_c = coarse.xyz[coarse.conn].mean(axis=1)
    cen_f = fine.xyz[fine.conn].mean(axis=1)
    for e in range(coarse.ne):
        j = int(np.argmin(((cen_f - cen_c[e]) ** 2).sum(1)))
        assert np.allclose(cen_f[j], cen_c[e], atol=1e-15)
        assert abs(phi_c[e] - phi_f[j]) < 1e-14


# --------------------------------------------------------------------------
# forward solve
# --------------------------------------------------------------------------
def _dense_imex(mesh, theta, dt, nsteps, v, w, a=0.1, eps=0.01, gamma=0.5):
    rp, ci, mv, kv = O.assemble(mesh, theta, SL, ST)
    M = O.csr_to_dense(rp, ci, mv, mesh.n)
    K = O.csr_to_dense(rp, ci, kv, mesh.n)
    lu = scipy.linalg.lu_factor(M + dt * K)
    v, w = v.copy(), w.copy()
    for _ in range(nsteps):
        R = v * (v - a) * (1 - v) - w
        vn = scipy.linalg.lu_solve(lu, M @ (v + dt * R))
        w = w + dt * eps * (v - gamma * w)
        v = vn
    return float(M.sum(axis=0) @ v), v, w


@pytest.mark.parametrize("m,dt,nsteps", [(3, 0.05, 20), (5, 0.1, 30)])
def test_solve_matches_dense_lu(m, dt, nsteps):
    mesh = O.mesh2d(m)
    rng = np.random.default_rng(m)
    theta = rng.normal(scale=0.8, size=mesh.ne)
    v0 = rng.uniform(0, 1, size=mesh.n)
    w0 = rng.uniform(0, 0.1, size=mesh.n)
    q, v, w, _, st = O.solve(mesh, theta, dt, nsteps, v0, w0)
    qd, vd, wd = _dense_imex(mesh, theta, dt, nsteps, v0, w0)
    assert st == 0
    assert abs(q - qd) < 1e-12 * abs(qd)
    assert np.max(np.abs(v - vd)) < 1e-11
    assert np.max(np.abs(w - wd)) < 1e-14


def test_solve_3d_matches_dense_lu():
    mesh = O.mesh3d(3, 3, 3, 1.0, 1.0, 0.25)
    rng = np.random.default_rng(7)
    theta = rng.normal(size=mesh.ne)
    v0 = rng.uniform(0, 1, size=mesh.n)
    w0 = np.zeros(mesh.n)
    q, v, _, _, st = O.solve(mesh, theta, 0.05, 10, v0, w0)
    qd, vd, _ = _dense_imex(mesh, theta, 0.05, 10, v0, w0)
    assert st == 0 and abs(q - qd) < 1e-12 * abs(qd) and np.max(np.abs(v - vd)) < 1e-11


def test_uniform_state_follows_scalar_recurrence():
    # K 1 = 0 and M (c 1) = c M 1: a spatially constant state evolves by the
    # scalar IMEX recurrence regardless of the fibre field.
    mesh = O.mesh2d(9)
    rng = np.random.default_rng(11)
    theta = rng.normal(size=mesh.ne)
    v, w = 0.6, 0.05
    dt, n = 0.05, 40
    q, vf, wf, _, st = O.solve(mesh, theta, dt, n, np.full(mesh.n, v), np.full(mesh.n, w))
    for _ in range(n):
        R = v * (v - 0.1) * (1 - v) - w
        v, w = v + dt * R, w + dt * 0.01 * (v - 0.5 * w)
    assert st == 0
    assert np.max(np.abs(vf - v)) < 1e-13 and np.max(np.abs(wf - w)) < 1e-15
    assert abs(q - v) < 1e-13                     # area of the unit square is 1


def test_one_block_conserves_mass_weighted_integral():
    # 1^T (M + dt K) = 1^T M, so m^T v+ = m^T (v + dt R) up to the residual.
    mesh = O.mesh2d(17)
    rng = np.random.default_rng(13)
    theta = rng.normal(size=mesh.ne)
    v0 = rng.uniform(0, 1, size=mesh.n)
    w0 = rng.uniform(0, 0.2, size=mesh.n)
    dt = 0.05
    q, *_ = O.solve(mesh, theta, dt, 1, v0, w0)
    rp, ci, mv, _ = O.assemble(mesh)
    mlump = O.csr_to_dense(rp, ci, mv, mesh.n).sum(axis=0)
    R = v0 * (v0 - 0.1) * (1 - v0) - w0
    assert abs(q - mlump @ (v0 + dt * R)) < 1e-13 * abs(q)


def test_mirror_symmetry():
    # Swapping x and y maps the mesh onto itself (lower <-> upper triangles)
    # and the fibre angle t onto pi/2 - t; the quarter-disc start is symmetric.
    m = 17
    mesh = O.mesh2d(m)
    rng = np.random.default_rng(17)
    theta = rng.normal(scale=0.5, size=mesh.ne)
    mirror = np.empty_like(theta)
    for j in range(m - 1):
        for i in range(m - 1):
            c, cm = i + (m - 1) * j, j + (m - 1) * i
            mirror[2 * cm + 1] = np.pi / 2 - theta[2 * c]
            mirror[2 * cm + 0] = np.pi / 2 - theta[2 * c + 1]
    q1 = O.solve(mesh, theta, 0.1, 30)[0]
    q2 = O.solve(mesh, mirror, 0.1, 30)[0]
    assert abs(q1 - q2) < 1e-11 * abs(q1)


def test_batch_equals_single_and_kl_synthesis():
    mesh = O.mesh2d(9)
    modes, _ = O.kl_build(mesh, 0.09, 0.04, 4)
    phi = O.centroid_table(mesh, modes, mesh)
    xi = inputs.gaussian_xi(0, 0, 0, 3, 4)
    q, it, st = O.solve_batch(mesh, phi, xi, 0.1, 10, nthreads=2)
    for s in range(3):
        theta = np.array([sum(phi[e, k] * xi[s, k] for k in range(4)) for e in range(mesh.ne)])
        qs = O.solve(mesh, theta, 0.1, 10)[0]
        assert abs(qs - q[s]) <= 1e-15 * abs(q[s])
    assert np.all(st == 0) and np.all(it > 0)


def test_solve_states_match_batch_and_qoi():
    # the per-sample field path: the same Q as the batched solver, and Q is
    # m^T v(T) with m = M 1 from the assembled consistent mass
    mesh = O.mesh2d(9)
    modes, _ = O.kl_build(mesh, 0.09, 0.04, 4)
    phi = O.centroid_table(mesh, modes, mesh)
    xi = inputs.gaussian_xi(0, 0, 0, 3, 4)
    tm = np.linspace(-0.2, 0.3, mesh.ne)
    q, it, st = O.solve_batch(mesh, phi, xi, 0.1, 10, theta_mean=tm, nthreads=2)
    qs, V, W, st2 = O.solve_states(mesh, phi, xi, 0.1, 10, theta_mean=tm)
    assert np.all(st2 == 0) and np.all(st == 0)
    # theta is summed in another order than in the batched C path: rounding only
    assert np.max(np.abs(qs - q) / np.abs(q)) <= 1e-13
    rp, ci, mv, _ = O.assemble(mesh)
    mvec = O.csr_to_dense(rp, ci, mv, mesh.n).sum(axis=1)
    assert np.allclose(V @ mvec, q, rtol=1e-14, atol=0)
    assert V.shape == (3, mesh.n) and np.all(np.isfinite(W)) and np.any(W != 0)


def test_maxiter_status():
    mesh = O.mesh2d(9)
    q, v, w, it, st = O.solve(mesh, np.zeros(mesh.ne), 0.1, 3, maxit=1)
    assert st == 1 and it == 3


# --------------------------------------------------------------------------
# estimators
# --------------------------------------------------------------------------
def test_mlmc_telescoping_on_common_samples():
    # sum_l (F_l - F_{l-1}) = F_L for every sample (eq. StandardML with the
    # same points on all levels), so the ML estimate equals the SL one.
    fine = O.mesh2d(17)
    modes, _ = O.kl_build(fine, 0.09, 0.04, 4)
    xi = inputs.gaussian_xi(0, 0, 0, 5, 4)
    meshes = [O.mesh2d(5), O.mesh2d(9), fine]
    dts = [0.2, 0.1, 0.05]
    q = [O.solve_batch(mm, O.centroid_table(fine, modes, mm), xi, dt, int(round(1.0 / dt)))[0]
         for mm, dt in zip(meshes, dts)]
    y = [q[0]] + [q[l] - q[l - 1] for l in (1, 2)]
    assert np.allclose(sum(y), q[2], rtol=1e-14, atol=0)
    est, var, _ = O.mlmc_estimate(y)
    assert abs(est - O.mc_estimate(q[2])[0]) < 1e-15


def test_mc_and_qmc_estimators_plain_definitions():
    q = np.array([1.0, 2.0, 4.0, 7.0])
    mean, var, rmse = O.mc_estimate(q)
    assert mean == 3.5 and abs(var - 7.0) < 1e-15 and abs(rmse - np.sqrt(7.0 / 4)) < 1e-15
    est, r = O.qmc_estimate(np.array([[1.0, 3.0], [2.0, 4.0], [3.0, 5.0]]))
    assert est == 3.0 and abs(r - 1.0 / np.sqrt(3)) < 1e-15


def test_cube_level_table_counts():
    # Table cube-levels of Sec. 5.2.1 (tests/golden/cube_levels.txt): h and
    # dt halve per level and the printed space-time DOF are 2^(4(l+1)).  With
    # the horizon T = 0.32 (not printed; the reading that makes the table
    # consistent) they equal the oracle's cube count of the Kuhn mesh of
    # [-0.5, 0.5]^3 at h_l times the number of time blocks T / dt_l.
    import os

    rows = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "cube_levels.txt"))
    T = 0.32
    for l, dof, h, dt in rows:
        l = int(l)
        assert h == 0.5 * 2.0 ** -l and abs(dt - 0.16 * 2.0 ** -l) < 1e-15
        m = int(round(1.0 / h)) + 1
        mesh = O.mesh3d(m, m, m, 1.0, 1.0, 1.0) if m <= 9 else None
        cubes = (m - 1) ** 3
        if mesh is not None:
            assert mesh.ne == 6 * cubes
            vol = np.abs(simplex_volumes(mesh))
            assert np.allclose(vol, h ** 3 / 6.0, rtol=1e-12)
        assert cubes * int(round(T / dt)) == int(dof)
        assert int(dof) == 2 ** (4 * (l + 1))


# --------------------------------------------------------------------------
# point QoIs of Sec. 2.4: action potential traces and activation times
# --------------------------------------------------------------------------
def test_activation_time_definition_on_hand_traces():
    dt, th = 0.1, 0.5
    assert O.activation_time(np.array([0.0, 0.2, 0.6, 0.9]), dt, th) == pytest.approx(0.1 + 0.1 * 0.3 / 0.4, abs=1e-15)
    assert O.activation_time(np.array([0.7, 0.2]), dt, th) == 0.0
    assert O.activation_time(np.array([0.0, 0.5]), dt, th) == pytest.approx(0.1, abs=1e-15)   # reached exactly
    assert O.activation_time(np.array([0.1, 0.4, 0.49]), dt, th) == -1.0


def test_point_traces_uniform_state_follow_scalar_recurrence():
    # a spatially constant state stays constant (K 1 = 0, M c1 = c M1): at
    # every point the trace is the scalar IMEX recurrence, and v0 = 0.3 > a
    # excites, so the trace crosses u_th and a(x0) lies on its linear piece
    mesh = O.mesh2d(9)
    K = 3
    modes, _ = O.kl_build(mesh, 0.09, 0.04, K)
    phi = O.centroid_table(mesh, modes, mesh)
    xi = inputs.gaussian_xi(2, 0, 0, 2, K)
    dt, nsteps, th = 0.2, 40, 0.5
    pts = np.array([[0.0, 0.0], [0.37, 0.81], [1.0, 0.5], [0.5, 0.5]])
    v0, w0 = np.full(mesh.n, 0.3), np.full(mesh.n, 0.01)
    tr, act, q, st = O.solve_points(mesh, phi, xi, dt, nsteps, pts, th, v0=v0, w0=w0)
    assert np.all(st == 0)
    a, eps, gam = 0.1, 0.01, 0.5
    v, w = 0.3, 0.01
    ref = [v]
    for _ in range(nsteps):
        v, w = v + dt * (v * (v - a) * (1 - v) - w), w + dt * eps * (v - gam * w)
        ref.append(v)
    ref = np.array(ref)
    assert np.max(np.abs(tr - ref[None, None, :])) < 1e-12
    n = int(np.argmax(ref >= th))
    assert n > 0 and ref[n - 1] < th <= ref[n]
    for s in range(2):
        for p in range(len(pts)):
            a_ = act[s, p]
            assert (n - 1) * dt < a_ <= n * dt + 1e-15
            u_at = tr[s, p, n - 1] + (a_ - (n - 1) * dt) / dt * (tr[s, p, n] - tr[s, p, n - 1])
            assert abs(u_at - th) < 1e-12


def test_point_traces_are_p1_values_of_the_state():
    # at a node the trace is the node's value; inside a triangle it is the
    # barycentric combination (weights from the geometry) of its vertices'
    # traces; the final entry matches solve_states' field
    m = 9
    h = 1.0 / (m - 1)
    mesh = O.mesh2d(m)
    K = 4
    modes, _ = O.kl_build(mesh, 0.09, 0.04, K)
    phi = O.centroid_table(mesh, modes, mesh)
    xi = inputs.gaussian_xi(5, 0, 0, 2, K)
    v0, w0 = O.initial_state(mesh, 0.35)
    i, j, s_, t_ = 3, 2, 0.7, 0.25                       # lower triangle of cell (3, 2): t <= s
    x = np.array([(i + s_) * h, (j + t_) * h])
    nodes = [(i, j), (i + 1, j), (i + 1, j + 1)]
    wts = [1 - s_, s_ - t_, t_]
    pts = np.vstack([x] + [np.array([a * h, b * h]) for a, b in nodes])
    dt, nsteps = 0.1, 12
    tr, act, q, st = O.solve_points(mesh, phi, xi, dt, nsteps, pts, 0.5, v0=v0, w0=w0)
    comb = sum(wt * tr[:, 1 + k, :] for k, wt in enumerate(wts))
    assert np.max(np.abs(tr[:, 0, :] - comb)) < 1e-14
    qs, V, W, _ = O.solve_states(mesh, phi, xi, dt, nsteps, v0=v0, w0=w0)
    for k, (a, b) in enumerate(nodes):
        assert np.array_equal(tr[:, 1 + k, -1], V[:, a + m * b])
    assert np.array_equal(q, qs)


def test_time_norms_match_quadrature_of_the_interpolant():
    import scipy.integrate

    rng = np.random.default_rng(4)
    T, nt = 2.5, 13
    e = rng.normal(size=nt + 1)
    t = np.linspace(0.0, T, nt + 1)
    l2, h1 = O.time_norms(e, T)
    f2 = sum(scipy.integrate.quad(lambda x: np.interp(x, t, e) ** 2, t[k], t[k + 1], epsabs=1e-14)[0]
             for k in range(nt))
    d2 = sum(((e[k + 1] - e[k]) / (t[k + 1] - t[k])) ** 2 * (t[k + 1] - t[k]) for k in range(nt))
    assert abs(l2 - np.sqrt(f2)) < 1e-12
    assert abs(h1 - np.sqrt(f2 + d2)) < 1e-12
    # a linear function: |e|_{H1}^2 = slope^2 T, ||e||^2 = T (e0^2 + e0 e1 + e1^2) / 3
    l2, h1 = O.time_norms(np.linspace(1.0, 3.0, 9), 2.0)
    assert abs(l2 ** 2 - 2.0 * (1 + 3 + 9) / 3) < 1e-12 and abs(h1 ** 2 - l2 ** 2 - 2.0) < 1e-12


# --------------------------------------------------------------------------
# the paper's scheme (eq. st-system, eq. mono_disc, eq. ionic_term)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("th", [0.5, 1.0])
def test_paper_scheme_linear_mode_amplification(th):
    # alpha = 0, no stimulus: an eigenvector K phi = lam M phi (scipy's
    # generalised eigensolver) is multiplied per block by the theta-scheme's
    # amplification factor (1 - (1 - theta) dt lam) / (1 + theta dt lam)
    mesh = O.mesh2d(7)
    tfield = np.full(mesh.ne, 0.4)
    rp, ci, mv, kv = O.assemble(mesh, tfield, SL, ST)
    M = O.csr_to_dense(rp, ci, mv, mesh.n)
    K = O.csr_to_dense(rp, ci, kv, mesh.n)
    lam, vec = scipy.linalg.eigh(K, M)
    j = 5
    phi = vec[:, j] / np.max(np.abs(vec[:, j]))
    dt, nb = 0.05, 7
    pm = dict(s_l=SL, s_t=ST, alpha=0.0, amp=0.0, theta=th)
    q, u, nw, st = O.solve_paper(mesh, tfield, dt, nb, u0=phi, pm=pm)
    rho = (1 - (1 - th) * dt * lam[j]) / (1 + th * dt * lam[j])
    assert st == 0
    assert np.max(np.abs(u - rho ** nb * phi)) < 1e-12


def test_paper_scheme_uniform_state_is_the_scalar_implicit_recurrence():
    # no stimulus and a constant state: K 1 = 0 and M c 1 = c M 1, so every
    # node follows u+ + dt I_ion(u+) = u (whatever theta), solved here by a
    # scalar Newton iteration
    mesh = O.mesh2d(9)
    tfield = np.linspace(-1.0, 1.0, mesh.ne)
    a, ur, uth, up = 1.4e-3, 0.0, 28.0, 115.0
    pm = dict(alpha=a, u_rest=ur, u_th=uth, u_peak=up, amp=0.0, theta=0.5)
    dt, nb = 0.05, 30
    q, u, nw, st = O.solve_paper(mesh, tfield, dt, nb, u0=np.full(mesh.n, 35.0), pm=pm)
    x = 35.0
    for _ in range(nb):
        y = x
        for _ in range(60):
            f = y + dt * a * (y - ur) * (y - uth) * (y - up) - x
            df = 1 + dt * a * ((y - uth) * (y - up) + (y - ur) * (y - up) + (y - ur) * (y - uth))
            y -= f / df
        x = y
    assert st == 0 and x > 35.0                     # above threshold: the cell activates
    assert np.max(np.abs(u - x)) < 1e-10 * x
    assert abs(q - x) < 1e-10 * x                   # |D| = 1


@pytest.mark.parametrize("th", [0.5, 1.0])
def test_paper_scheme_block_balance(th):
    # summing the block equations (1^T K = 0): m^T u+ + dt m^T I_ion(u+) =
    # m^T u + dt m^T (theta g(t+) + (1 - theta) g(t)), g the nodal stimulus;
    # a slip in the reaction's sign or time level, or in the stimulus weights,
    # breaks it
    mesh = O.mesh2d(9)
    rp, ci, mv, _ = O.assemble(mesh)
    m = O.csr_to_dense(rp, ci, mv, mesh.n).sum(axis=1)
    rng = np.random.default_rng(8)
    tfield = rng.normal(size=mesh.ne)
    u0 = rng.uniform(0, 60, mesh.n)
    pm = dict(theta=th, sigma=0.3, t1=0.15, amp=115.0, x0=(0.2, 0.3))
    p = O._paper_vec(pm)
    dt = 0.1
    q, u1, nw, st = O.solve_paper(mesh, tfield, dt, 1, u0=u0, pm=pm)
    ion = lambda u: p[2] * (u - p[3]) * (u - p[4]) * (u - p[5])
    g = lambda t: (p[3] + p[7] * np.exp(-np.sum((mesh.xyz - p[10:12]) ** 2, axis=1) / p[8] ** 2)) * (t < p[9])
    lhs = m @ u1 + dt * m @ ion(u1)
    rhs = m @ u0 + dt * m @ (th * g(dt) + (1 - th) * g(0.0))
    assert st == 0 and abs(lhs - rhs) < 1e-11 * abs(rhs)


def test_five_level_fixture_reproduces_from_the_oracle():
    # tests/golden/mlmc_2d_5levels_oracle_y.txt was written by its script
    # from the oracle alone: its first samples of levels 0 and 1 come out of
    # the oracle again bit for bit (the oracle's per-sample arithmetic does
    # not depend on the batch or the thread count), and its estimate and
    # variances are eq. StandardML of its own Y_l
    import os

    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "mlmc_2d_5levels_oracle_y.txt")
    head, ys = {}, []
    for line in open(path):
        w = line.split()
        if line.startswith("#"):
            continue
        if w[0] in ("estimate", "var", "rmse"):
            head[w[0]] = [float(x) for x in w[1:]]
        elif w[0] == "level":
            ys.append([])
        else:
            ys[-1].append(float(w[0]))
    ys = [np.array(y) for y in ys]
    assert [y.size for y in ys] == [4096, 1024, 256, 64, 16]
    est, var, rmse = O.mlmc_estimate(ys)
    assert est == head["estimate"][0] and rmse == head["rmse"][0]
    assert np.array_equal(var, head["var"])
    fine = O.mesh2d(257)
    modes, _ = O.kl_build(fine, 0.09, 0.04, 16)
    m17, m33 = O.mesh2d(17), O.mesh2d(33)
    p17, p33 = O.centroid_table(fine, modes, m17), O.centroid_table(fine, modes, m33)
    xi0 = inputs.gaussian_xi(0, 0, 0, 3, 16)
    assert np.array_equal(O.solve_batch(m17, p17, xi0, 0.1, 100)[0], ys[0][:3])
    xi1 = inputs.gaussian_xi(0, 1, 0, 2, 16)
    y1 = O.solve_batch(m33, p33, xi1, 0.05, 200)[0] - O.solve_batch(m17, p17, xi1, 0.1, 100)[0]
    assert np.array_equal(y1, ys[1][:2])
