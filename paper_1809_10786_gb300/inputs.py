"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module draws random numbers and nothing else: it holds none of the
transform's arithmetic, so both the CUDA path and the CPU oracle can be fed from
it without sharing any code of the method.

Distributions follow the workloads of the paper's experiments as restated for
this library (coefficients and values uniform in a complex square, points from
the Gaussian weight exp(-|x|^2), i.e. N(0, I/2), kept inside the ball of radius 5
used in Sect. 8).  Seeds are ``1809_10786 + 1000 * workload + instance``.
"""
import math

import numpy as np

SEED_BASE = 1809_10786
RMAX = 5.0


def seed_for(workload, instance=0):
    return SEED_BASE + 1000 * int(workload) + int(instance)


def num_coeffs(B):
    return B * (B + 1) * (2 * B + 1) // 6


def degree_of_index(B):
    """Array n(mu) for mu = 0..Nc-1 (layout only: n outer, then l, then m)."""
    out = np.empty(num_coeffs(B), dtype=np.int64)
    pos = 0
    for n in range(1, B + 1):
        out[pos:pos + n * n] = n
        pos += n * n
    return out


def coefficients(B, seed, half_width=0.5, scale_by_degree=False):
    """complex128 [Nc], real and imaginary parts uniform in [-half_width, half_width]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nc = num_coeffs(B)
    c = rng.uniform(-half_width, half_width, nc) + 1j * rng.uniform(-half_width, half_width, nc)
    if scale_by_degree:
        c = c / degree_of_index(B)
    return c.astype(np.complex128)


def points_gaussian(M, seed, rmax=RMAX):
    """float64 [M, 3] ~ N(0, I/2) (density prop. to exp(-|x|^2)), rejection to |x| <= rmax."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = np.empty((M, 3), dtype=np.float64)
    got = 0
    while got < M:
        x = rng.normal(0.0, math.sqrt(0.5), size=(max(M - got, 16) + 16, 3))
        x = x[np.einsum("ij,ij->i", x, x) <= rmax * rmax]
        take = min(M - got, x.shape[0])
        out[got:got + take] = x[:take]
        got += take
    return out


def points_ball(M, seed, radius=RMAX):
    """float64 [M, 3] uniform in the ball of the given radius (the paper's Sect. 8 points)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    d = rng.normal(size=(M, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = radius * rng.uniform(0.0, 1.0, M) ** (1.0 / 3.0)
    return (d * r[:, None]).astype(np.float64)


def values(M, seed, half_width=0.5):
    """complex128 [M], real and imaginary parts uniform in [-half_width, half_width]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return (rng.uniform(-half_width, half_width, M) + 1j * rng.uniform(-half_width, half_width, M)).astype(np.complex128)


def complex_normal(M, seed, scale=1.0):
    """complex128 [M]: scale * (a + i b)/sqrt(2), a, b ~ N(0, 1)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return (scale * (rng.normal(size=M) + 1j * rng.normal(size=M)) / math.sqrt(2.0)).astype(np.complex128)


def subset(M, k, seed):
    """First k indices of a seeded permutation of range(M) (oracle subsets)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.sort(rng.permutation(M)[:min(k, M)])


def batch_instances(n, seed, b_lo=8, b_hi=48, m_lo_exp=3.0, m_hi_exp=5.0):
    """n independent (B, M) pairs: B uniform in {b_lo..b_hi}, M = round(10^U[m_lo_exp, m_hi_exp])."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Bs = rng.integers(b_lo, b_hi + 1, size=n)
    Ms = np.rint(10.0 ** rng.uniform(m_lo_exp, m_hi_exp, size=n)).astype(np.int64)
    return [(int(b), int(m)) for b, m in zip(Bs, Ms)]
