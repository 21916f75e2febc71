"""The seeded input recipe (CPU only): every generator is deterministic in its seed and draws
the distribution it states -- points N(0, I/2) kept in |x| <= 5 or uniform in a ball,
coefficients and values uniform in a complex square, the batch workload's (B, M) pairs."""
import math

import numpy as np
import pytest

from paper_1809_10786_gb300 import inputs


def test_seeds_are_distinct_per_workload_and_instance():
    seeds = {inputs.seed_for(w, i) for w in range(5) for i in range(1000)}
    assert len(seeds) == 5000


@pytest.mark.parametrize("gen,args", [(inputs.points_gaussian, (5000,)), (inputs.points_ball, (5000,)),
                                      (inputs.values, (5000,)), (inputs.complex_normal, (5000,)),
                                      (inputs.coefficients, (12,))])
def test_generators_are_deterministic_in_their_seed(gen, args):
    a, b, c = gen(*args, 11), gen(*args, 11), gen(*args, 12)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, c)


def test_gaussian_points_follow_the_weight_exp_minus_r2():
    M = 200_000
    x = inputs.points_gaussian(M, 3)
    assert x.shape == (M, 3) and x.dtype == np.float64
    r2 = np.einsum("ij,ij->i", x, x)
    assert r2.max() <= inputs.RMAX ** 2
    # N(0, I/2): each coordinate has variance 1/2 (the cut at r = 5 removes a 1e-10 tail), and
    # |x|^2 is Gamma(3/2, 1): P(|x|^2 <= 1) = erf(1) - 2 e^{-1} / sqrt(pi)
    assert np.allclose(x.var(axis=0), 0.5, rtol=0.02)
    assert np.allclose(x.mean(axis=0), 0.0, atol=0.01)
    p1 = math.erf(1.0) - 2.0 * math.exp(-1.0) / math.sqrt(math.pi)
    assert abs(np.mean(r2 <= 1.0) - p1) < 0.005


def test_rejection_keeps_every_point_inside_a_small_radius():
    x = inputs.points_gaussian(20_000, 4, rmax=1.0)
    assert x.shape == (20_000, 3)
    assert np.einsum("ij,ij->i", x, x).max() <= 1.0


@pytest.mark.parametrize("radius", [1.0, 5.0])
def test_ball_points_are_uniform_in_the_ball(radius):
    M = 100_000
    x = inputs.points_ball(M, 5, radius=radius)
    r = np.linalg.norm(x, axis=1)
    assert r.max() <= radius * (1 + 1e-12)
    # uniform in the ball: P(r <= s R) = s^3
    for s in (0.3, 0.5, 0.8):
        assert abs(np.mean(r <= s * radius) - s ** 3) < 0.006
    # and isotropic
    assert np.allclose((x / r[:, None]).mean(axis=0), 0.0, atol=0.01)


def test_coefficients_fill_the_complex_square():
    B = 20
    c = inputs.coefficients(B, 6)
    assert c.shape == (inputs.num_coeffs(B),) and c.dtype == np.complex128
    assert np.abs(c.real).max() <= 0.5 and np.abs(c.imag).max() <= 0.5
    assert abs(c.real.var() - 1.0 / 12.0) < 0.005 and abs(c.imag.var() - 1.0 / 12.0) < 0.005
    # the degree scaling divides entry mu by n(mu)
    s = inputs.coefficients(B, 6, scale_by_degree=True)
    assert np.allclose(s * inputs.degree_of_index(B), c)


def test_coefficient_layout_counts_n_squared_entries_per_degree():
    for B in (1, 2, 7, 64):
        n = inputs.degree_of_index(B)
        assert len(n) == inputs.num_coeffs(B) == sum(k * k for k in range(1, B + 1))
        assert all(np.count_nonzero(n == k) == k * k for k in range(1, B + 1))
        assert np.all(np.diff(n) >= 0)


def test_values_and_complex_normals():
    v = inputs.values(50_000, 7)
    assert v.dtype == np.complex128 and np.abs(v.real).max() <= 0.5 and np.abs(v.imag).max() <= 0.5
    z = inputs.complex_normal(200_000, 8, scale=2.0)
    assert abs(np.mean(np.abs(z) ** 2) - 4.0) < 0.05          # E|z|^2 = scale^2


def test_subset_draws_distinct_sorted_indices():
    s = inputs.subset(1000, 100, 9)
    assert len(s) == 100 and len(np.unique(s)) == 100 and np.all(np.diff(s) > 0)
    assert s.min() >= 0 and s.max() < 1000
    assert np.array_equal(inputs.subset(10, 100, 9), np.arange(10))     # k > M: all of them


def test_batch_workload_pairs():
    pairs = inputs.batch_instances(256, inputs.seed_for(3))
    assert len(pairs) == 256
    Bs = np.array([b for b, _ in pairs])
    Ms = np.array([m for _, m in pairs])
    assert Bs.min() >= 8 and Bs.max() <= 48 and len(np.unique(Bs)) > 30
    assert Ms.min() >= 1000 and Ms.max() <= 100_000
    # log10 M uniform on [3, 5]: about half of the instances below 10^4
    assert 0.35 < np.mean(Ms < 10_000) < 0.65
