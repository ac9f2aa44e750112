"""Seeded sample points: the only module both the CUDA path and the oracle use.

It holds none of the method's arithmetic.  It turns (seed, level, sample
index) into the random variables xi that parametrise the fibre field
(eq. KLlowrank), so that both sides see bit-identical inputs:

* Monte Carlo: xi ~ N(0,1) from the counter-based Philox4x32-10 generator
  (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
  SC'11) and the Box-Muller transform (Box & Muller 1958).  Counter =
  (sample, pair index, level, stream), key = (seed, 0): a sample's variables
  do not depend on how many samples are drawn or in which batch.
* Quasi-Monte Carlo: a randomly shifted rank-1 lattice rule
  y_i = frac(i z / N + Delta), xi = Phi^{-1}(y), with the generating vector z
  chosen component by component (Sloan & Reztsov 2002; Nuyens & Cools 2006)
  for product weights gamma_k, and shifts Delta from Philox.
* Halton points (Halton 1960): coordinate k of point i is the radical
  inverse of i in the k-th prime base.  With the paper's uniform random
  variables Y_k on [-1, 1] (Sec. 2.3: sigma_k = sqrt(3 lambda_k)) a point maps
  to xi_k = sqrt(3) (2 y_k - 1), the unit-variance scaling of the modes.
"""
from __future__ import annotations

import math

import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr: np.ndarray, key: np.ndarray) -> np.ndarray:
    """Philox4x32 with 10 rounds.  ctr: (..., 4) uint32, key: (..., 2) uint32.
    Returns (..., 4) uint32."""
    c = np.asarray(ctr, dtype=np.uint64) & _MASK
    k = np.asarray(key, dtype=np.uint64) & _MASK
    c0, c1, c2, c3 = c[..., 0], c[..., 1], c[..., 2], c[..., 3]
    k0, k1 = k[..., 0].copy(), k[..., 1].copy()
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
        p0 = _M0 * c0          # < 2^64: both factors < 2^32
        p1 = _M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & _MASK, lo1, (hi0 ^ c3 ^ k1) & _MASK, lo0
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


def _u53(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Two 32-bit words -> a double in (0, 1) with 53 random bits."""
    hi = (a.astype(np.uint64) >> np.uint64(5)).astype(np.float64)   # 27 bits
    lo = (b.astype(np.uint64) >> np.uint64(6)).astype(np.float64)   # 26 bits
    return (hi * 67108864.0 + lo + 0.5) / 9007199254740992.0


def gaussian_xi(seed: int, level: int, first: int, count: int, K: int, stream: int = 0) -> np.ndarray:
    """xi[s, k] ~ N(0,1) for samples first..first+count-1 of a level:
    one Philox block per (sample, pair of k), Box-Muller on the two
    uniforms it yields.  Shape (count, K), float64."""
    npair = (K + 1) // 2
    s = np.arange(first, first + count, dtype=np.uint64)
    j = np.arange(npair, dtype=np.uint64)
    ctr = np.zeros((count, npair, 4), dtype=np.uint64)
    ctr[..., 0] = s[:, None] & _MASK
    ctr[..., 1] = j[None, :]
    ctr[..., 2] = np.uint64(level)
    ctr[..., 3] = np.uint64(stream)
    key = np.zeros((count, npair, 2), dtype=np.uint64)
    key[..., 0] = np.uint64(seed) & _MASK
    key[..., 1] = (np.uint64(seed) >> np.uint64(32)) & _MASK
    w = philox4x32_10(ctr, key)
    u1 = _u53(w[..., 0], w[..., 1])
    u2 = _u53(w[..., 2], w[..., 3])
    rad = np.sqrt(-2.0 * np.log(u1))
    z = np.empty((count, 2 * npair))
    z[:, 0::2] = rad * np.cos(2.0 * np.pi * u2)
    z[:, 1::2] = rad * np.sin(2.0 * np.pi * u2)
    return np.ascontiguousarray(z[:, :K])


def uniform_shifts(seed: int, level: int, R: int, K: int, stream: int = 1) -> np.ndarray:
    """R random shifts in [0,1)^K for a lattice rule, from Philox."""
    nq = (K + 1) // 2
    r = np.arange(R, dtype=np.uint64)
    j = np.arange(nq, dtype=np.uint64)
    ctr = np.zeros((R, nq, 4), dtype=np.uint64)
    ctr[..., 0] = r[:, None]
    ctr[..., 1] = j[None, :]
    ctr[..., 2] = np.uint64(level)
    ctr[..., 3] = np.uint64(stream)
    key = np.zeros((R, nq, 2), dtype=np.uint64)
    key[..., 0] = np.uint64(seed) & _MASK
    w = philox4x32_10(ctr, key)
    u = np.empty((R, 2 * nq))
    u[:, 0::2] = _u53(w[..., 0], w[..., 1])
    u[:, 1::2] = _u53(w[..., 2], w[..., 3])
    return np.ascontiguousarray(u[:, :K] - 0.5 / 9007199254740992.0)


def _bernoulli2(x: np.ndarray) -> np.ndarray:
    return x * x - x + 1.0 / 6.0


def cbc_lattice(N: int, K: int, gamma: np.ndarray) -> np.ndarray:
    """Generating vector of an N-point rank-1 lattice rule, built component by
    component: z_k minimises the shift-averaged worst-case error
        e^2(z) = -1 + (1/N) sum_i prod_k (1 + gamma_k 2 pi^2 B2({i z_k / N}))
    over z_k in {1 <= z < N, gcd(z, N) = 1}, earlier components fixed."""
    gamma = np.asarray(gamma, dtype=np.float64)
    cand = np.array([z for z in range(1, max(N, 2)) if math.gcd(z, N) == 1], dtype=np.int64)
    if N == 1:
        return np.ones(K, dtype=np.int64)
    i = np.arange(N, dtype=np.int64)
    prod = np.ones(N)
    z = np.zeros(K, dtype=np.int64)
    frac = ((i[None, :] * cand[:, None]) % N) / N                  # (candidates, N)
    omega = 2.0 * np.pi ** 2 * _bernoulli2(frac)
    for k in range(K):
        err = (prod[None, :] * (1.0 + gamma[k] * omega)).mean(axis=1)
        best = int(np.argmin(err))
        z[k] = cand[best]
        prod = prod * (1.0 + gamma[k] * omega[best])
    return z


def lattice_points(z: np.ndarray, N: int, shift: np.ndarray) -> np.ndarray:
    """y_i = frac(i z / N + shift), i = 0..N-1.  Shape (N, K)."""
    i = np.arange(N, dtype=np.int64)[:, None]
    y = ((i * np.asarray(z)[None, :]) % N) / N + np.asarray(shift)[None, :]
    return y - np.floor(y)


def gaussian_from_uniform(y: np.ndarray) -> np.ndarray:
    """xi = Phi^{-1}(y); y = 0 is mapped to 2^-53 first."""
    from scipy.special import ndtri

    y = np.where(y <= 0.0, 2.0 ** -53, y)
    return ndtri(y)


def qmc_xi(seed: int, level: int, N: int, R: int, K: int, gamma: np.ndarray) -> np.ndarray:
    """Shifted-lattice sample points for one level: shape (R, N, K)."""
    z = cbc_lattice(N, K, gamma)
    shifts = uniform_shifts(seed, level, R, K)
    return np.stack([gaussian_from_uniform(lattice_points(z, N, shifts[r])) for r in range(R)])


def first_primes(K: int) -> np.ndarray:
    """The first K primes."""
    out = []
    c = 2
    while len(out) < K:
        if all(c % p for p in out if p * p <= c):
            out.append(c)
        c += 1
    return np.array(out, dtype=np.int64)


def radical_inverse(i: np.ndarray, base: int) -> np.ndarray:
    """sum_j d_j base^-(j+1) for i = sum_j d_j base^j (exact in base 2, to
    rounding in the other bases)."""
    i = np.asarray(i, dtype=np.int64).copy()
    out = np.zeros(i.shape, dtype=np.float64)
    f = 1.0 / base
    while np.any(i > 0):
        out += (i % base) * f
        i //= base
        f /= base
    return out


def halton(N: int, K: int, first: int = 0) -> np.ndarray:
    """Points first .. first + N - 1 of the K-dimensional Halton sequence.
    Shape (N, K), entries in [0, 1).  Point 0 is the origin, which
    uniform_xi maps to the corner xi = -sqrt(3) in every coordinate: an
    unrandomised quadrature rule should start at first = 1 so that it does
    not carry that corner sample (first = 0 keeps the exact stratification
    of the first b^m points in base b)."""
    idx = np.arange(first, first + N, dtype=np.int64)
    return np.stack([radical_inverse(idx, int(b)) for b in first_primes(K)], axis=1)


def uniform_xi(y: np.ndarray) -> np.ndarray:
    """xi = sqrt(3) (2 y - 1): Y uniform on [-1, 1] with unit variance."""
    return math.sqrt(3.0) * (2.0 * np.asarray(y, dtype=np.float64) - 1.0)
