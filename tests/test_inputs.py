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
