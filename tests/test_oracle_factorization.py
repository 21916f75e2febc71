"""Pins of the factorization and NFFT oracles.

* The factorization of Lambda (Sect. 6 theorem) is exact: the NDFT of eta at the
  transformed points equals the direct sum (Sect. 7, first sentence; the exact
  NDFT control of Sect. 8, fourth test).
* eta lives on |k0| <= 2B-2, |k1| <= B-1, |k2| <= B-1 (degrees stated in Sect. 6),
  is even in k0 (beta_{-kappa} = beta_kappa) and has the parity of m in k1.
* The Gaussian NFFT obeys the bound of the Thm. on the d-dimensional NFFT error.
* The window Fourier pairs hold (Lemma on the Gaussian transform; the
  Kaiser-Bessel pair checked by quadrature).
* The paper's printed error order at q = 16 (Sect. 8, first test) is reproduced.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import direct, factorization as fz, nfft
from paper_1809_10786_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_sect8.json")


def _case(B, M, seed):
    c = inputs.coefficients(B, seed)
    x = inputs.points_gaussian(M, seed + 1)
    rho = float(np.linalg.norm(x, axis=1).max())
    return c, x, rho


@pytest.mark.parametrize("B,M", [(2, 50), (8, 400), (13, 300)])
def test_factorization_is_exact(B, M):
    c, x, rho = _case(B, M, 100 + B)
    f, _ = direct.forward(B, x, c)
    eta = fz.eta(B, c, rho)
    g = fz.ndft(eta, fz.torus_points(x, rho))
    assert np.abs(g - f).max() <= 1e-12 * np.abs(f).max()


def test_factorization_valid_for_any_rho_above_max_radius():
    # the factorization holds for every rho >= max r_i (Sect. 6 choice of rho)
    B = 7
    c, x, rho = _case(B, 200, 7)
    f, _ = direct.forward(B, x, c)
    for r in (rho, 1.3 * rho, 2.0 * rho):
        g = fz.ndft(fz.eta(B, c, r), fz.torus_points(x, r))
        assert np.abs(g - f).max() <= 1e-11 * np.abs(f).max()


def test_eta_support_and_symmetries():
    B = 9
    c, x, rho = _case(B, 10, 9)
    eta = fz.eta(B, c, rho)
    scale = np.abs(eta).max()
    k = np.arange(4 * B) - 2 * B
    K0, K1, K2 = np.meshgrid(k, k, k, indexing="ij")
    outside = (np.abs(K0) > 2 * B - 2) | (np.abs(K1) > B - 1) | (np.abs(K2) > B - 1)
    assert np.abs(eta[outside]).max() <= 1e-13 * scale
    # even in k0
    for a in range(1, 2 * B - 1):
        assert np.abs(eta[2 * B + a] - eta[2 * B - a]).max() <= 1e-13 * scale
    # parity of m in k1
    for m in range(-(B - 1), B):
        s = 1 if m % 2 == 0 else -1
        for b in range(1, B):
            d = eta[:, 2 * B + b, 2 * B + m] - s * eta[:, 2 * B - b, 2 * B + m]
            assert np.abs(d).max() <= 1e-13 * scale


def test_ndft_of_single_frequency():
    cube = np.zeros((6, 4, 8), dtype=np.complex128)
    cube[3 + 2, 2 - 1, 4 + 3] = 2.0 - 1.0j
    t = np.array([[0.3, 1.1, 5.9], [2.0, 0.1, 0.0]])
    g = fz.ndft(cube, t)
    ref = (2.0 - 1.0j) * np.exp(1j * (2 * t[:, 0] - 1 * t[:, 1] + 3 * t[:, 2]))
    assert np.abs(g - ref).max() < 1e-14


@pytest.mark.parametrize("q", [2, 4, 6, 8, 10])
def test_gauss_nfft_within_theorem_bound(q):
    B = 6
    c, x, rho = _case(B, 300, 200 + q)
    eta = fz.eta(B, c, rho)
    om = eta[:, B:3 * B, B:3 * B]               # the 4B x 2B x 2B grid of Sect. 8
    t = fz.torus_points(x, rho)
    exact = fz.ndft(om, t)
    s = nfft.nfft(om, t, 2.0, q, "gauss")
    err = np.abs(s - exact).max()
    assert err <= nfft.gauss_error_bound(3, 2.0, q) * np.abs(om).sum()


def test_kb_beats_gauss_and_decays():
    B = 6
    c, x, rho = _case(B, 300, 300)
    eta = fz.eta(B, c, rho)
    om = eta[:, B:3 * B, B:3 * B]
    t = fz.torus_points(x, rho)
    exact = fz.ndft(om, t)
    errs = []
    for q in (2, 3, 4, 5, 6):
        ekb = np.abs(nfft.nfft(om, t, 2.0, q, "kb") - exact).max()
        ega = np.abs(nfft.nfft(om, t, 2.0, q, "gauss") - exact).max()
        assert ekb < ega
        errs.append(ekb)
    assert all(b < 0.2 * a for a, b in zip(errs, errs[1:]))


@pytest.mark.parametrize("window", ["gauss", "kb"])
@pytest.mark.parametrize("q", [4, 8])
def test_window_fourier_pairs_by_quadrature(window, q):
    # int psi(xi) e^{-i kappa xi} d xi over the truncated support against the closed form
    N, sigma = 64, 2.0
    xg, wg = np.polynomial.legendre.leggauss(400)
    a = 2 * math.pi * q / N
    xi = a * xg
    psi = nfft.window_value(xi, N, sigma, q, window)
    for kappa in (0, 3, 11, 16):
        quad = a * np.sum(wg * psi * np.cos(kappa * xi))
        ref = nfft.window_fourier(kappa, N, sigma, q, window)
        # the untruncated pair differs from the truncated integral by the window tails
        # (Gaussian: exp(-q^2/(2 lam)) scale; Kaiser-Bessel: exp(-b q) relative to the peak)
        tail = 2e-3 if window == "gauss" else max(10 * math.exp(-nfft.kb_shape(sigma) * q), 1e-12)
        assert abs(quad - ref) <= tail * abs(ref) + 1e-14


def test_gauss_fourier_matches_lemma_closed_form():
    # Lemma: int phi(x) e^{-i<k,x>} dx = prod exp(-2 lam (pi kappa / sigma n)^2); integrate the
    # untruncated 1-D Gaussian of the Def. on a wide interval
    N, sigma, q = 32, 2.0, 6
    lam = nfft.gauss_lambda(sigma, q)
    xs = np.linspace(-math.pi, math.pi, 20001)
    u = N * xs / (2 * math.pi)
    phi = (N / (2 * math.pi)) / math.sqrt(2 * math.pi * lam) * np.exp(-u * u / (2 * lam))
    for kappa in (0, 2, 7):
        quad = np.trapezoid(phi * np.cos(kappa * xs), xs)
        assert abs(quad - math.exp(-2 * lam * (math.pi * kappa / N) ** 2)) < 1e-10


@pytest.mark.slow
def test_paper_error_order_at_q16():
    # Sect. 8 first test: B = 32, sigma = 2, q = 16, points uniform in the ball of radius 5,
    # coefficients uniform in [-1,1]^2: relative error on the order of 1e-10.
    gold = json.load(open(GOLDEN))["error_test"]
    B, M = 32, 120
    c = inputs.coefficients(B, 4242, half_width=1.0)
    x = inputs.points_ball(M, 4243, radius=5.0)
    rho = float(np.linalg.norm(x, axis=1).max())
    f, _ = direct.forward(B, x, c)
    eta = fz.eta(B, c, rho)
    om = eta[:, B:3 * B, B:3 * B]
    s = nfft.nfft(om, fz.torus_points(x, rho), gold["sigma"], gold["q"], "gauss")
    rel = np.max(np.abs(s - f) / np.abs(f))
    order = gold["relative_error_order"]
    assert order / 1e3 < rel < order * 1e3, rel
