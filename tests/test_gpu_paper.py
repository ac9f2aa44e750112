"""The paper's time discretization (Sec. 3.1 eq. st-system with the reaction
of eq. mono_disc on the new time level, the current of eq. ionic_term with
the paper's constants, the stimulus of Sec. 5.1) through the C ABI, against
the oracle, which solves each block by Newton's method with the full
Jacobian and BiCGSTAB; the library runs chord-Newton sweeps with CG on
M + theta dt K.  Both converge to the root of the same block system, so
they agree to the solver tolerances: FP64 1e-10, mixed 1e-6 (relative per
sample on Q, and relative to max |u| on the field u(T))."""
import numpy as np
import pytest

import oracle as O
from paper_2105_02007_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 1: 1e-6}
# slower diffusion than the configurations' so that the stimulated front
# travels across the square within T = 4
MODEL = dict(s_l=0.01, s_t=0.002)


@pytest.fixture(scope="module")
def mlq():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_02007_gb300 import build

    build.build()
    from paper_2105_02007_gb300 import mlq as m

    return m


@pytest.mark.parametrize("theta", [0.5, 1.0])
@pytest.mark.parametrize("prec,storage", [(0, 0), (1, 0), (1, 2)])
def test_paper_scheme_parity(mlq, theta, prec, storage):
    m, K, S, dt, nb = 33, 6, 3, 0.02, 200
    mesh = O.mesh2d(m)
    modes, _ = O.kl_build(mesh, 0.09, 0.04, K)
    phi = O.centroid_table(mesh, modes, mesh)
    xi = inputs.gaussian_xi(50, 0, 0, S, K)
    pm = dict(MODEL, theta=theta, sigma=0.2, t1=1.0)
    q_ref, U_ref, st = O.solve_paper_batch(mesh, phi, xi, dt, nb, pm=pm)
    assert np.all(st == 0)
    assert np.max(U_ref) > 100.0                      # the stimulus excited a front
    with mlq.Context(0, prec, storage=storage) as ctx:
        ctx.set_model(**MODEL)
        ctx.set_scheme(ionic=1, theta=theta, sigma=0.2, t1=1.0)
        ctx.add_level(0, m, dt, nb)
        ctx.set_kl(0, phi)
        r = ctx.solve_state(0, xi)
    assert np.all(r["status"] == 0), r["status"]
    assert np.max(np.abs(r["q"] - q_ref) / np.abs(q_ref)) < TOL[prec]
    assert np.max(np.abs(r["v"] - U_ref)) < TOL[prec] * np.max(np.abs(U_ref))


def test_paper_scheme_rejects_3d(mlq):
    with mlq.Context(0, mlq.MLQ_MIXED) as ctx:
        ctx.add_level(0, (5, 5, 3), 0.05, 2)
        with pytest.raises(mlq.MLQError) as e:
            ctx.set_scheme(ionic=1, theta=0.5)
        assert e.value.code == -6
    with mlq.Context(0, mlq.MLQ_MIXED) as ctx:
        ctx.set_scheme(ionic=1, theta=0.5)
        with pytest.raises(mlq.MLQError):
            ctx.add_level(0, (5, 5, 3), 0.05, 2)
