"""Point quantities of interest of Sec. 2.4 (action potential u(x0, t) and
activation time a(x0)), formed inside the solvers' block loops, against the
oracle on the same seeded inputs.

Traces are compared element by element relative to max |u| with the solver
tolerances (FP64 1e-10, mixed 1e-6).  An activation time is a crossing
t_{n-1} + dt (u_th - u_{n-1}) / (u_n - u_{n-1}); a perturbation du of the
trace moves it by about dt du / (u_n - u_{n-1}), which is the bound used.
Where the two sides put the first block with u_n >= u_th at different n
(floating point deciding an integer), the test checks that the trace there
lies within the tolerance of u_th, so both choices are valid.
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


def check_points(r, tr, act, dt, th, tol):
    scale = np.max(np.abs(tr))
    assert np.max(np.abs(r["trace"] - tr)) <= tol * scale
    S, P = act.shape
    for s in range(S):
        for p in range(P):
            a_g, a_o = r["act"][s, p], act[s, p]
            u = tr[s, p]
            if (a_g < 0) != (a_o < 0) or (a_g >= 0 and int(np.ceil(a_g / dt - 1e-9)) != int(np.ceil(a_o / dt - 1e-9))):
                # different crossing blocks: the trace must sit at the threshold there
                n = int(np.argmin(np.abs(u - th)))
                assert abs(u[n] - th) <= 10 * tol * scale, (s, p, a_g, a_o)
                continue
            if a_o < 0:
                continue
            n = max(1, int(np.ceil(a_o / dt - 1e-9)))
            du = max(u[n] - u[n - 1], 1e-300)
            assert abs(a_g - a_o) <= dt * 4 * tol * scale / du + 1e-12, (s, p, a_g, a_o)


@pytest.mark.parametrize("prec,precond", [(0, 0), (1, 0), (1, 1)])
def test_points_2d_parity(mlq, prec, precond):
    # slower diffusion than the configurations' (s_l = 0.01, s_t = 0.002) so
    # that the excitation travels across the square within T = 30
    m, K, S, dt, nsteps, th = 33, 8, 6, 0.5, 60, 0.5
    model = dict(s_l=0.01, s_t=0.002)
    mesh = O.mesh2d(m)
    modes, _ = O.kl_build(mesh, 0.09, 0.04, K)
    phi = O.centroid_table(mesh, modes, mesh)
    xi = inputs.gaussian_xi(21, 0, 0, S, K)
    pts = np.array([[0.0, 0.0], [0.5, 0.5], [0.31, 0.12], [0.12, 0.43], [0.6, 0.2], [1.0, 1.0], [0.45, 0.45]])
    v0, w0 = O.initial_state(mesh, 0.3)
    tr, act, q, st = O.solve_points(mesh, phi, xi, dt, nsteps, pts, th, v0=v0, w0=w0, model=model)
    assert np.all(st == 0)
    assert np.sum(act > 0) >= S * 3 and np.any(act < 0)    # most points activate, the far corner does not
    with mlq.Context(0, prec, precond=precond) as ctx:
        ctx.set_model(**model)
        ctx.add_level(0, m, dt, nsteps)
        ctx.set_kl(0, phi)
        ctx.set_initial_disk(0, 0.3)
        ctx.set_points(0, pts, th)
        r = ctx.solve_points(0, xi)
        plain = ctx.solve(0, xi)
    assert np.all(r["status"] == 0)
    assert np.array_equal(r["q"], plain["q_fine"])            # the points do not change the solve
    check_points(r, tr, act, dt, th, TOL[prec])


@pytest.mark.parametrize("prec,precond", [(0, 0), (1, 1)])
def test_points_3d_parity(mlq, prec, precond):
    dims, K, S, dt, nsteps, th = (9, 9, 5), 6, 3, 0.5, 40, 0.5
    model = dict(s_l=0.01, s_t=0.002)
    mesh = O.mesh3d(*dims)
    modes, _ = O.kl_build(mesh, 0.09, 0.15 ** 2, K)
    phi = O.centroid_table(mesh, modes, mesh)
    xi = inputs.gaussian_xi(22, 0, 0, S, K)
    pts = np.array([[0.0, 0.0, 0.0], [0.21, 0.13, 0.05], [0.5, 0.3, 0.2], [0.3, 0.3, 0.1], [0.9, 0.1, 0.25]])
    v0, w0 = O.initial_state(mesh, 0.35)
    tr, act, q, st = O.solve_points(mesh, phi, xi, dt, nsteps, pts, th, v0=v0, w0=w0, model=model)
    assert np.all(st == 0)
    assert np.sum(act > 0) >= S
    with mlq.Context(0, prec, precond=precond) as ctx:
        ctx.set_model(**model)
        ctx.add_level(0, dims, dt, nsteps)
        ctx.set_kl(0, phi)
        ctx.set_initial_disk(0, 0.35)
        ctx.set_points(0, pts, th)
        r = ctx.solve_points(0, xi)
    assert np.all(r["status"] == 0)
    check_points(r, tr, act, dt, th, TOL[prec])


def test_points_rejected_outside_and_level_difference(mlq):
    # a point outside the domain is refused; the level difference of a trace
    # QoI (fine trace minus the prolonged coarse one) goes to zero in H1(0,T)
    # under refinement of the pair
    with mlq.Context(0, mlq.MLQ_MIXED) as ctx:
        ctx.add_level(0, 17, 0.1, 20)
        with pytest.raises(mlq.MLQError):
            ctx.set_points(0, np.array([[1.2, 0.5]]), 0.5)
    fine = O.mesh2d(65)
    modes, _ = O.kl_build(fine, 0.09, 0.04, 6)
    xi = inputs.gaussian_xi(23, 0, 0, 2, 6)
    pts = np.array([[0.25, 0.25]])
    T = 8.0
    diffs = []
    with mlq.Context(0, mlq.MLQ_MIXED) as ctx:
        ctx.set_model(s_l=0.01, s_t=0.002)
        for l, m in enumerate([17, 33, 65]):
            dt = 0.4 * 0.5 ** l
            ctx.add_level(l, m, dt, int(round(T / dt)))
            ctx.set_kl(l, O.centroid_table(fine, modes, O.mesh2d(m)))
            ctx.set_initial_disk(l, 0.3)
            ctx.set_points(l, pts, 0.5)
        tr = [ctx.solve_points(l, xi)["trace"] for l in range(3)]
    for l in (1, 2):
        d = [mlq.time_norms(tr[l][s, 0] - mlq.trace_prolong(tr[l - 1][s, 0]), T)[1] for s in range(2)]
        diffs.append(max(d))
    assert diffs[1] < diffs[0]
