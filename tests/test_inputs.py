"""The seeded sample-point generators shared by both sides."""
import os

import numpy as np

from paper_2105_02007_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = inputs.philox4x32_10(np.array(v[:4], dtype=np.uint32), np.array(v[4:6], dtype=np.uint32))
        assert [int(x) for x in out] == v[6:]


def test_gaussian_xi_counter_based_and_moments():
    a = inputs.gaussian_xi(0, 2, 0, 40, 7)
    b = inputs.gaussian_xi(0, 2, 10, 5, 7)
    assert np.array_equal(a[10:15], b)                       # batch independent
    assert not np.array_equal(inputs.gaussian_xi(0, 3, 0, 4, 7), a[:4])
    z = inputs.gaussian_xi(0, 0, 0, 20000, 16).ravel()
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1) < 0.01
    assert abs(np.mean(z ** 4) - 3) < 0.05


def test_lattice_integrates_trig_polynomials_exactly():
    N, K = 64, 5
    gamma = 1.0 / np.arange(1, K + 1) ** 2
    z = inputs.cbc_lattice(N, K, gamma)
    assert np.all(np.gcd(z, N) == 1)
    y = inputs.lattice_points(z, N, np.zeros(K))
    rng = np.random.default_rng(0)
    for _ in range(50):
        h = rng.integers(-3, 4, size=K)
        s = np.exp(2j * np.pi * (y @ h)).mean()
        if int(h @ z) % N == 0:
            assert abs(s - 1) < 1e-12                        # on the dual lattice
        else:
            assert abs(s) < 1e-12                            # integrated exactly (to 0)


def test_cbc_beats_random_vector():
    N, K = 61, 4
    gamma = np.array([1.0, 0.5, 0.25, 0.125])

    def err(z):
        i = np.arange(N)[:, None]
        x = (i * z[None, :] % N) / N
        return np.mean(np.prod(1 + gamma * 2 * np.pi ** 2 * (x * x - x + 1 / 6), axis=1)) - 1

    zc = inputs.cbc_lattice(N, K, gamma)
    rng = np.random.default_rng(1)
    rand = [err(rng.integers(1, N, size=K)) for _ in range(20)]
    assert err(zc) <= min(rand) + 1e-15


def test_qmc_xi_shapes_and_shift_range():
    x = inputs.qmc_xi(0, 1, 16, 4, 3, np.ones(3))
    assert x.shape == (4, 16, 3) and np.all(np.isfinite(x))
    s = inputs.uniform_shifts(0, 1, 100, 3)
    assert s.min() >= 0 and s.max() < 1


def test_halton_known_points_and_stratification():
    from paper_2105_02007_gb300 import inputs

    assert list(inputs.first_primes(6)) == [2, 3, 5, 7, 11, 13]
    h = inputs.halton(9, 3)
    assert list(h[:5, 0]) == [0.0, 0.5, 0.25, 0.75, 0.125]
    assert np.allclose(h[:4, 1], [0.0, 1 / 3, 2 / 3, 1 / 9], rtol=0, atol=1e-15)
    assert np.allclose(h[1:6, 2], [0.2, 0.4, 0.6, 0.8, 0.04], rtol=0, atol=1e-15)
    # the first b^m points of coordinate k are the grid {j / b^m} (exactly in
    # base 2, to rounding in the others)
    for k, b in enumerate([2, 3, 5]):
        m = {2: 10, 3: 6, 5: 4}[b]
        col = np.sort(inputs.halton(b ** m, 3)[:, k])
        if b == 2:
            assert np.array_equal(col, np.arange(b ** m) / b ** m)
        else:
            assert np.max(np.abs(col - np.arange(b ** m) / b ** m)) < 1e-15
    # consecutive blocks continue the sequence
    assert np.array_equal(inputs.halton(5, 4, first=7), inputs.halton(12, 4)[7:])


def test_halton_integrates_better_than_random_points():
    from paper_2105_02007_gb300 import inputs

    K = 3
    f = lambda y: np.prod(1.0 + 0.5 * (y - 0.5), axis=1)     # exact integral 1
    err = [abs(f(inputs.halton(N, K)).mean() - 1.0) for N in (1024, 16384)]
    # close to the 1/N rate of a low-discrepancy sequence (random points: 1/sqrt N)
    assert err[1] < err[0] / 8
    rng = np.random.default_rng(0)
    err_mc = np.sqrt(np.mean([(f(rng.random((16384, K))).mean() - 1.0) ** 2 for _ in range(20)]))
    assert err[1] < err_mc / 5


def test_uniform_map_has_unit_variance():
    from paper_2105_02007_gb300 import inputs

    # on the grid {j / N} the map gives exactly mean -sqrt(3)/N and the
    # variance of the discrete uniform law on N points of [-sqrt 3, sqrt 3)
    N = 2 ** 12
    xi = inputs.uniform_xi(np.arange(N) / N)
    assert abs(xi.mean() + np.sqrt(3.0) / N) < 1e-14
    assert abs(xi.var() - (1.0 - 1.0 / N ** 2)) < 1e-12
    assert xi.min() == -np.sqrt(3.0) and xi.max() < np.sqrt(3.0)
