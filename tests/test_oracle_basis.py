"""Pins of the direct-summation oracle against closed forms and identities the
paper's definitions fix (Sect. 1 definition of H_nlm, Thm. on completeness and
orthonormality, Sect. 4 Legendre recurrence, Sect. 7 Legendre identities)."""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import direct
from paper_1809_10786_gb300 import inputs

PI = math.pi


def sph(x):
    r = np.linalg.norm(x)
    return r, math.acos(x[2] / r), math.atan2(x[1], x[0])


def test_coefficient_count_and_index_roundtrip():
    for B in (1, 2, 5, 8, 33):
        assert direct.num_coeffs(B) == B * (B + 1) * (2 * B + 1) // 6
    mu = 0
    for n in range(1, 9):
        for l in range(n):
            for m in range(-l, l + 1):
                assert direct.mu(n, l, m) == mu
                assert direct.nlm(mu) == (n, l, m)
                mu += 1


def test_index_closed_form_agrees_away_from_zero():
    # Sect. 1 closed form n(mu) = floor(cosh(arcosh(36 sqrt3 mu)/3)/sqrt3 + 1/2) is read only for mu >= 1
    # (arcosh is undefined at 0); the oracle uses a search.
    # At the first index of each n-block the real-arithmetic value is the integer n itself, and
    # double rounding may land just below it; everywhere else the floor is unambiguous.
    for mu_ in range(1, 2000):
        v = math.cosh(math.acosh(36 * math.sqrt(3) * mu_) / 3) / math.sqrt(3) + 0.5
        n, l, m = direct.nlm(mu_)
        if mu_ == n * (n - 1) * (2 * n - 1) // 6:
            assert abs(v - n) < 1e-9
        else:
            assert math.floor(v) == n
        rem = mu_ - n * (n - 1) * (2 * n - 1) // 6
        assert math.isqrt(rem) == l and rem - l * (l + 1) == m


@pytest.mark.parametrize("x", [(0.3, -0.2, 0.5), (-1.1, 0.4, 2.0), (0.05, 0.07, -0.3)])
def test_low_order_closed_forms(x):
    x = np.array(x)
    h = direct.basis(4, x)
    r2 = float(x @ x)
    # H_100 = N_10 Y_00 = pi^{-3/4}
    assert abs(h[direct.mu(1, 0, 0)] - PI ** -0.75) < 1e-15
    # H_200 = N_20 L_1^{(1/2)}(r^2) Y_00, N_20 = sqrt(2/Gamma(5/2)), L_1^{(a)}(x) = 1 + a - x
    N20 = math.sqrt(2 / math.gamma(2.5))
    assert abs(h[direct.mu(2, 0, 0)] - N20 * (1.5 - r2) / math.sqrt(4 * PI)) < 1e-14
    # H_300 with L_2^{(a)}(x) = (x^2 - 2(a+2)x + (a+1)(a+2))/2
    N30 = math.sqrt(2 * 2 / math.gamma(3.5))
    L2 = (r2 * r2 - 2 * 2.5 * r2 + 1.5 * 2.5) / 2
    assert abs(h[direct.mu(3, 0, 0)] - N30 * L2 / math.sqrt(4 * PI)) < 1e-14
    # H_21m = N_21 r Y_1m, Y_10 = sqrt(3/4pi) cos t, Y_11 = -sqrt(3/8pi) sin t e^{i phi}, Y_1-1 = -conj(Y_11)
    N21 = math.sqrt(2 / math.gamma(2.5))
    assert abs(h[direct.mu(2, 1, 0)] - N21 * math.sqrt(3 / (4 * PI)) * x[2]) < 1e-15
    y11 = -math.sqrt(3 / (8 * PI)) * (x[0] + 1j * x[1])
    assert abs(h[direct.mu(2, 1, 1)] - N21 * y11) < 1e-15
    assert abs(h[direct.mu(2, 1, -1)] - N21 * (-np.conj(y11))) < 1e-15
    # H_322 = N_32 r^2 Y_22, Y_22 = (1/4) sqrt(15/(2 pi)) sin^2 t e^{2 i phi}
    N32 = math.sqrt(2 / math.gamma(3.5))
    y22 = 0.25 * math.sqrt(15 / (2 * PI)) * (x[0] + 1j * x[1]) ** 2
    assert abs(h[direct.mu(3, 2, 2)] - N32 * y22) < 1e-14


def _laguerre_exact(k, a, x):
    # explicit sum L_k^{(a)}(x) = sum_i (-1)^i binom(k+a, k-i) x^i / i!, exact in rationals
    tot = Fraction(0)
    for i in range(k + 1):
        num = Fraction(1)
        for j in range(k - i):            # binom(k+a, k-i) = prod_{j<k-i} (a+i+1+j)/(j+1)
            num *= (a + i + 1 + j) / Fraction(j + 1)
        tot += (-1) ** i * num * x ** i / math.factorial(i)
    return tot


@pytest.mark.parametrize("a2,x", [(1, Fraction(3, 4)), (7, Fraction(5, 2)), (21, Fraction(9, 1))])
def test_laguerre_against_exact_rational_sum(a2, x):
    a = Fraction(a2, 2)
    K = 24
    got = direct.laguerre(K, float(a), float(x))
    for k in range(K + 1):
        ex = float(_laguerre_exact(k, a, x))
        assert abs(got[k] - ex) <= 1e-12 * max(1.0, abs(ex)), (k, got[k], ex)


def test_addition_theorem_and_rotation_invariance():
    # sum_m |Y_lm|^2 = (2l+1)/(4pi)  =>  sum_m |H_nlm(x)|^2 = |H_nl0(r e_z)|^2 (Y_l0(0) = sqrt((2l+1)/4pi))
    B = 12
    rng = np.random.default_rng(3)
    for _ in range(5):
        x = rng.normal(size=3)
        r = np.linalg.norm(x)
        h = direct.basis(B, x)
        hz = direct.basis(B, np.array([0.0, 0.0, r]))
        for n in range(1, B + 1):
            for l in range(n):
                s = sum(abs(h[direct.mu(n, l, m)]) ** 2 for m in range(-l, l + 1))
                ref = abs(hz[direct.mu(n, l, 0)]) ** 2
                assert abs(s - ref) <= 1e-10 * ref + 1e-15
                for m in range(-l, l + 1):
                    if m != 0:
                        assert abs(hz[direct.mu(n, l, m)]) < 1e-13


def test_parity():
    B = 10
    x = np.array([0.7, -0.4, 1.3])
    h, hm = direct.basis(B, x), direct.basis(B, -x)
    for mu_ in range(direct.num_coeffs(B)):
        n, l, m = direct.nlm(mu_)
        assert abs(hm[mu_] - (-1) ** l * h[mu_]) < 1e-12 * max(1, abs(h[mu_]))


@pytest.mark.parametrize("B", [3, 5])
def test_orthonormality_by_exact_quadrature(B):
    # <H, H'> with weight exp(-|x|^2): generalized Gauss-Laguerre (alpha = 1/2) in t = r^2,
    # Gauss-Legendre in cos(theta), equispaced phi; exact for bandwidth B (Thm. on completeness).
    from scipy.special import roots_genlaguerre
    tq, wt = roots_genlaguerre(B + 1, 0.5)
    xq, wx = np.polynomial.legendre.leggauss(B + 1)
    nphi = 2 * B + 1
    phis = 2 * PI * np.arange(nphi) / nphi
    Nc = direct.num_coeffs(B)
    G = np.zeros((Nc, Nc), dtype=np.complex128)
    for t, w1 in zip(tq, wt):
        r = math.sqrt(t)
        for ct, w2 in zip(xq, wx):
            st = math.sqrt(1 - ct * ct)
            for ph in phis:
                x = r * np.array([st * math.cos(ph), st * math.sin(ph), ct])
                h = direct.basis(B, x)
                # int_0^inf f r^2 e^{-r^2} dr = (1/2) int_0^inf f t^{1/2} e^{-t} dt
                G += (0.5 * w1 * w2 * (2 * PI / nphi)) * np.outer(h, np.conj(h))
    assert np.abs(G - np.eye(Nc)).max() < 1e-12


def test_real_symmetric_coefficients_give_real_values():
    B = 8
    c = inputs.coefficients(B, 11)
    for n in range(1, B + 1):
        for l in range(n):
            c[direct.mu(n, l, 0)] = c[direct.mu(n, l, 0)].real
            for m in range(1, l + 1):
                c[direct.mu(n, l, -m)] = (-1) ** m * np.conj(c[direct.mu(n, l, m)])
    x = inputs.points_gaussian(50, 12)
    f, _ = direct.forward(B, x, c)
    assert np.abs(f.imag).max() < 1e-13 * np.abs(f.real).max()


def test_rotation_about_z():
    B = 9
    c = inputs.coefficients(B, 21)
    x = inputs.points_gaussian(40, 22)
    phi0 = 0.7
    R = np.array([[math.cos(phi0), -math.sin(phi0), 0], [math.sin(phi0), math.cos(phi0), 0], [0, 0, 1]])
    m_of = np.array([direct.nlm(k)[2] for k in range(direct.num_coeffs(B))])
    f_rot, _ = direct.forward(B, x @ R.T, c)
    f_c, _ = direct.forward(B, x, c * np.exp(1j * m_of * phi0))
    assert np.abs(f_rot - f_c).max() < 1e-12 * np.abs(f_c).max()


def test_adjoint_identity():
    B = 10
    c = inputs.coefficients(B, 31)
    x = inputs.points_gaussian(300, 32)
    y = inputs.values(300, 33)
    f, _ = direct.forward(B, x, c)
    a, _ = direct.adjoint(B, x, y)
    lhs = np.vdot(y, f)          # <Lambda c, y> = sum conj(y) (Lambda c)
    rhs = np.vdot(a, c)          # <c, Lambda^H y> = sum conj(Lambda^H y) c
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(f) * np.linalg.norm(y)


def test_threads_do_not_change_results():
    B = 7
    c = inputs.coefficients(B, 41)
    x = inputs.points_gaussian(97, 42)
    y = inputs.values(97, 43)
    f1, t1 = direct.forward(B, x, c, nthreads=1)
    f4, t4 = direct.forward(B, x, c, nthreads=4)
    assert t1 == 1 and t4 == 4
    assert np.array_equal(f1, f4)
    a1, _ = direct.adjoint(B, x, y, nthreads=1)
    a4, _ = direct.adjoint(B, x, y, nthreads=4)
    assert np.abs(a1 - a4).max() < 1e-13 * np.abs(a1).max()


def test_gradient_against_central_differences():
    B = 8
    c = inputs.coefficients(B, 51)
    x = inputs.points_gaussian(25, 52)
    g = inputs.values(25, 53)
    grad, _ = direct.grad_points(B, x, c, g)
    h = 1e-6
    fd = np.zeros_like(grad)
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        fp, _ = direct.forward(B, x + e, c)
        fm, _ = direct.forward(B, x - e, c)
        fd[:, d] = np.real(np.conj(g) * (fp - fm) / (2 * h))
    assert np.abs(grad - fd).max() <= 1e-6 * np.abs(fd).max()


def test_gradient_near_axis_and_origin_is_finite_and_consistent():
    # points close to the z-axis and to the origin: the spherical-coordinate
    # singularities are removed by the identities of Sect. 7
    B = 6
    c = inputs.coefficients(B, 61)
    x = np.array([[1e-9, 2e-9, 0.8], [0.3, -0.2, 1e-10], [1e-7, -1e-7, 1e-7], [0.0, 0.0, -1.2]])
    g = np.ones(4, dtype=np.complex128)
    grad, _ = direct.grad_points(B, x, c, g)
    assert np.all(np.isfinite(grad))
    h = 1e-6
    for i in range(2):
        for d in range(3):
            e = np.zeros(3)
            e[d] = h
            fp, _ = direct.forward(B, x[i:i + 1] + e, c)
            fm, _ = direct.forward(B, x[i:i + 1] - e, c)
            fd = np.real((fp - fm) / (2 * h))[0]
            assert abs(grad[i, d] - fd) <= 1e-6 * max(1, abs(fd))


@pytest.mark.slow
def test_long_double_build_agrees():
    # the same source rounded in a wider type: agreement bounds the oracle's own rounding error
    B = 48
    c = inputs.coefficients(B, 71)
    x = inputs.points_gaussian(6, 72)
    x[0] *= 4.5 / np.linalg.norm(x[0])          # include a far point (r = 4.5)
    f, _ = direct.forward(B, x, c)
    fl, _ = direct.forward(B, x, c, kind="long double")
    assert direct.real_bytes("long double") > 8
    assert np.abs(f - fl).max() <= 1e-12 * np.abs(fl).max()
