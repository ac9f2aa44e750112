"""Estimators on top of the batched solver (Sec. 4): the adaptive multilevel
Monte Carlo driver (pilot samples, variances, sample allocation of eq.
StandardML, top-up) and a field-valued QoI (the state v_h(T)) with the
nested intergrid transfer, against the oracle on the same seeded inputs."""
import os

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


MS, DTS, T, K = [9, 17, 33], [0.2, 0.1, 0.05], 4.0, 4


def hierarchy():
    fine = O.mesh2d(MS[-1])
    modes, _ = O.kl_build(fine, 0.09, 0.04, K)
    meshes = [O.mesh2d(m) for m in MS]
    return meshes, [O.centroid_table(fine, modes, mm) for mm in meshes]


def test_adaptive_mlmc_meets_the_allocation_and_matches_the_oracle(mlq):
    meshes, phis = hierarchy()
    pools = [inputs.gaussian_xi(31, l, 0, n, K) for l, n in enumerate([1200, 400, 120])]
    eps = 2e-7
    with mlq.Context(0, mlq.MLQ_MIXED) as ctx:
        for l, (m, dt, ph) in enumerate(zip(MS, DTS, phis)):
            ctx.add_level(l, m, dt, int(round(T / dt)))
            ctx.set_kl(l, ph)
        N, mean, var, rmse = ctx.estimate_adaptive(pools, eps, n_pilot=16)
        # the same numbers from direct solves of the first N_l samples of each pool
        ys = [ctx.solve(l, pools[l][: N[l]], with_coarse=l > 0)["y"] for l in range(3)]
        again = ctx.estimate_adaptive(pools, eps, n_pilot=16)
    assert np.all(N >= 16) and np.all(N <= [1200, 400, 120])
    assert np.any(N > 16)                                      # the pilot was topped up
    assert rmse <= eps or np.any(N == [1200, 400, 120])
    m2, v2, r2 = mlq.mlmc_combine(ys)
    assert m2 == mean and r2 == rmse and np.array_equal(v2, var)
    assert np.array_equal(again[0], N) and again[1] == mean            # deterministic
    # the allocation for the final variances is met (the loop's exit rule)
    cost = [MS[l] ** 2 * round(T / DTS[l]) + (MS[l - 1] ** 2 * round(T / DTS[l - 1]) if l else 0) for l in range(3)]
    alloc = mlq.mlmc_allocation(var, np.array(cost, dtype=float), eps, 16)
    assert np.all((alloc <= N) | (N == np.array([1200, 400, 120])))
    # parity: the oracle's level differences of the same samples
    yo = []
    for l in range(3):
        qf = O.solve_batch(meshes[l], phis[l], pools[l][: N[l]], DTS[l], int(round(T / DTS[l])), nthreads=4)[0]
        qc = (O.solve_batch(meshes[l - 1], phis[l - 1], pools[l][: N[l]], DTS[l - 1], int(round(T / DTS[l - 1])),
                            nthreads=4)[0] if l else 0.0)
        yo.append(qf - qc)
    mo, vo, ro = O.mlmc_estimate(yo)
    assert abs(mean - mo) <= 1e-6 * abs(mo)
    assert abs(rmse - ro) <= 1e-4 * ro


def test_field_qoi_multilevel_mean_matches_the_oracle(mlq):
    # E[v(T)] on the 33 x 33 mesh by eq. StandardML over two levels: the mean
    # of v_0 prolonged, plus the mean of Y_1 = v_1 - P v_0 (same xi)
    meshes, phis = hierarchy()
    xi0 = inputs.gaussian_xi(32, 1, 0, 24, K)
    xi1 = inputs.gaussian_xi(32, 2, 0, 8, K)
    with mlq.Context(0, mlq.MLQ_MIXED) as ctx:
        for l in (1, 2):
            ctx.add_level(l, MS[l], DTS[l], int(round(T / DTS[l])))
            ctx.set_kl(l, phis[l])
        v0 = ctx.solve_state(1, xi0)["v"]
        f1 = ctx.solve_state(2, xi1)["v"]
        c1 = ctx.solve_state(1, xi1)["v"]
    P = lambda v: mlq.field_prolong(MS[1], v)
    mean = np.mean([P(v) for v in v0], axis=0) + np.mean([f - P(c) for f, c in zip(f1, c1)], axis=0)
    # the oracle: its own states and its point location for the transfer
    V0 = O.solve_states(meshes[1], phis[1], xi0, DTS[1], int(round(T / DTS[1])))[1]
    F1 = O.solve_states(meshes[2], phis[2], xi1, DTS[2], int(round(T / DTS[2])))[1]
    C1 = O.solve_states(meshes[1], phis[1], xi1, DTS[1], int(round(T / DTS[1])))[1]
    Po = lambda v: O.p1_at_points(meshes[1], v[:, None], meshes[2].xyz)[:, 0]
    ref = np.mean([Po(v) for v in V0], axis=0) + np.mean([f - Po(c) for f, c in zip(F1, C1)], axis=0)
    err = mlq.field_norms(MS[2], mean - ref)[0]
    assert err <= 1e-6 * mlq.field_norms(MS[2], ref)[0]
    # the level difference is small against the field in H1(D)
    y1 = np.mean([f - P(c) for f, c in zip(f1, c1)], axis=0)
    assert mlq.field_norms(MS[2], y1)[1] < mlq.field_norms(MS[2], mean)[1]


def test_five_level_estimate_with_the_coarsest_members_merged(mlq):
    # five levels give nine members on eight lanes: the two members on the
    # coarsest mesh (pair 0's fine, pair 1's coarse) run as one launch; each
    # sample must come out exactly as in its own member (mlq_solve per
    # level), and the estimate as eq. StandardML of the oracle's solves
    ms, dts, T5 = [5, 9, 17, 33, 65], [0.4, 0.2, 0.1, 0.05, 0.025], 2.0
    N = [48, 24, 12, 6, 4]
    fine = O.mesh2d(ms[-1])
    modes, _ = O.kl_build(fine, 0.09, 0.04, K)
    meshes = [O.mesh2d(m) for m in ms]
    phis = [O.centroid_table(fine, modes, mm) for mm in meshes]
    xis = [inputs.gaussian_xi(46, l, 0, N[l], K) for l in range(5)]
    with mlq.Context(0, mlq.MLQ_MIXED) as ctx:
        for l, (m, dt, ph) in enumerate(zip(ms, dts, phis)):
            ctx.add_level(l, m, dt, int(round(T5 / dt)))
            ctx.set_kl(l, ph)
        ctx.set_profiling(True)
        mean, var, rmse, ys = ctx.estimate(xis, return_y=True)
        members = ctx.member_profile()
        ctx.set_profiling(False)
        direct = [ctx.solve(l, xis[l], with_coarse=l > 0)["y"] for l in range(5)]
    # eight launches: the 5^2 mesh's two members ran as one of N_0 + N_1 samples
    assert len(members) == 8
    assert any(m["level"] == 0 and m["samples"] == N[0] + N[1] for m in members)
    for l in range(5):
        assert np.array_equal(ys[l], direct[l]), l
    yref = []
    for l in range(5):
        qf = O.solve_batch(meshes[l], phis[l], xis[l], dts[l], int(round(T5 / dts[l])), nthreads=4)[0]
        qc = (O.solve_batch(meshes[l - 1], phis[l - 1], xis[l], dts[l - 1], int(round(T5 / dts[l - 1])),
                            nthreads=4)[0] if l else 0.0)
        yref.append(qf - qc)
    est_ref = sum(float(np.mean(y)) for y in yref)
    assert abs(mean - est_ref) <= 1e-6 * abs(est_ref)


def read_five_level_golden():
    """(estimate, V_l, [Y_l per sample]) of tests/golden/mlmc_2d_5levels_oracle_y.txt."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "mlmc_2d_5levels_oracle_y.txt")
    est, var, ys = None, None, []
    with open(path) as f:
        for line in f:
            if line.startswith("#"):
                continue
            w = line.split()
            if w[0] == "estimate":
                est = float(w[1])
            elif w[0] == "var":
                var = [float(x) for x in w[1:]]
            elif w[0] == "level":
                ys.append([])
            elif w[0] != "rmse":
                ys[-1].append(float(w[0]))
    return est, var, [np.array(y) for y in ys]


def test_full_five_level_estimate_matches_the_oracle_sample_by_sample(mlq):
    # the whole five-level 2D workload (17^2 .. 257^2 nodes, 4096 / 1024 /
    # 256 / 64 / 16 samples, K = 16, dt_l = 0.1 2^-l over T = 10) in the
    # mixed path, fed the oracle's KL tables: every sample's Y_l against the
    # oracle's (tests/golden, written from the oracle alone over every
    # sample and the whole horizon).  Each Q within 1e-6 relative bounds a
    # Y_l within d = 2e-6 max |Q|; max |Q| is taken from the level-0 values,
    # which are Q_0 (the coarsest mesh gives the largest Q here), with a 1 %
    # margin
    est_ref, var_ref, ys_ref = read_five_level_golden()
    ms, N = [17, 33, 65, 129, 257], [4096, 1024, 256, 64, 16]
    assert [y.size for y in ys_ref] == N
    fine = O.mesh2d(ms[-1])
    modes, _ = O.kl_build(fine, 0.09, 0.04, 16)
    phis = [O.centroid_table(fine, modes, O.mesh2d(m)) for m in ms]
    xis = [inputs.gaussian_xi(0, l, 0, N[l], 16) for l in range(5)]
    with mlq.Context(0, mlq.MLQ_MIXED) as ctx:
        for l, m in enumerate(ms):
            ctx.add_level(l, m, 0.1 * 0.5 ** l, 100 * 2 ** l)
            ctx.set_kl(l, phis[l])
        mean, var, rmse, ys = ctx.estimate(xis, return_y=True)
    d = 2e-6 * 1.01 * float(np.max(np.abs(ys_ref[0])))
    for l in range(5):
        assert np.max(np.abs(ys[l] - ys_ref[l])) <= d, l
        # each deviation from the mean moves by at most 2 d, so the unbiased
        # sample variance moves by at most (4 d sum |y_i - m| + 4 d^2 n) /
        # (n - 1) <= (4 d sqrt(n (n - 1) V) + 4 d^2 n) / (n - 1)
        n = N[l]
        assert abs(var[l] - var_ref[l]) <= (4 * d * np.sqrt(n * (n - 1) * var_ref[l]) + 4 * d * d * n) / (n - 1)
    assert abs(mean - est_ref) <= 5 * d
