"""Pins of the inverse-transform oracle (CPU): CGNR / CGNE against closed forms.

CG on the normal equations reaches, in exact arithmetic, the least-squares solution (first
kind, M >= Nc) or the minimum-norm solution (second kind, M < Nc) within Nc, resp. M, steps:
numpy's lstsq gives both in closed form.  The mid-point-rule initial guess of the paper's last
test is pinned by the orthonormality of the SGL basis under the weight e^{-|x|^2}.
"""
import numpy as np
import pytest

from oracle import direct, inverse
from paper_1809_10786_gb300 import inputs


def points_in_ball(M, seed, radius):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((M, 3))
    v /= np.linalg.norm(v, axis=1)[:, None]
    return v * radius * rng.random(M)[:, None] ** (1 / 3)


def test_cgnr_reaches_least_squares_solution():
    B, M = 3, 80
    L = inverse.matrix(B, points_in_ball(M, 11, 2.0))
    f = L @ inputs.coefficients(B, 12) + 1e-3 * inputs.complex_normal(M, 13)     # inconsistent system
    c_ls = np.linalg.lstsq(L, f, rcond=None)[0]
    c, res = inverse.cgnr(L, f, np.zeros(L.shape[1], complex), iters=4 * L.shape[1])
    assert np.abs(c - c_ls).max() <= 1e-8 * np.abs(c_ls).max()
    # CGNR minimizes the residual over growing Krylov spaces: non-increasing
    assert all(b <= a * (1 + 1e-12) for a, b in zip(res, res[1:]))
    assert res[-1] == pytest.approx(np.linalg.norm(f - L @ c_ls), rel=1e-9)


def test_cgne_reaches_minimum_norm_solution():
    B, M = 4, 18                                  # Nc = 30 > M
    L = inverse.matrix(B, points_in_ball(M, 21, 1.5))
    f = inputs.complex_normal(M, 22)
    c_mn = np.linalg.lstsq(L, f, rcond=None)[0]   # minimum-norm solution for full row rank
    c, res = inverse.cgne(L, f, np.zeros(L.shape[1], complex), iters=4 * M)
    assert np.abs(c - c_mn).max() <= 1e-8 * np.abs(c_mn).max()
    assert res[-1] <= 1e-9 * res[0]


def test_matrix_columns_are_the_basis_and_match_the_direct_sums():
    B, M = 3, 7
    x = points_in_ball(M, 31, 2.0)
    L = inverse.matrix(B, x)
    c = inputs.coefficients(B, 32)
    f, _ = direct.forward(B, x, c)
    assert np.abs(L @ c - f).max() <= 1e-13 * np.abs(f).max()
    y = inputs.complex_normal(M, 33)
    a, _ = direct.adjoint(B, x, y)
    assert np.abs(L.conj().T @ y - a).max() <= 1e-13 * np.abs(a).max()


def test_midpoint_guess_integrates_with_the_orthonormality_weight():
    # f = H_mu for one mu: the rule h^3 sum f conj(H_nu) e^{-|x|^2} approximates the inner
    # product <H_mu, H_nu> = delta_{mu nu} (the integrand decays like e^{-|x|^2} at the box edge)
    B, N, kappa = 2, 48, 5.0
    x = inverse.cartesian_grid(N, kappa)
    assert x.shape == (N ** 3, 3) and x.min() == -kappa and x.max() == pytest.approx(kappa * (1 - 2.0 / N))
    Nc = direct.num_coeffs(B)
    for mu in range(Nc):
        e = np.zeros(Nc, complex)
        e[mu] = 1.0
        f, _ = direct.forward(B, x, e)
        g = inverse.midpoint_guess(B, x, f, kappa, N)
        assert np.abs(g - e).max() <= 1e-6
