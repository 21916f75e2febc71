"""Error-driven choice of the NFFT cutoff (CPU; the bound is host code).

The only approximating step of the transform is the final NFFT (Sect. 7, error estimate), so
max |f - f~| <= bound * ||eta||_1.  The library computes the bound from its own window, cutoff and
grid; the oracle computes the same definition with its independent window pair and NFFT steps.
Pins: agreement with the oracle; the paper's closed-form Gaussian bound (Thm. on the NFFT error)
is never below it; on the oracle's own 3-D NFFT the measured errors stay below it.
"""
import ctypes
import json
import math
import os

import numpy as np
import pytest

from oracle import nfft
from paper_1809_10786_gb300 import binding

KB, GAUSS = 0, 1
NAMES = {KB: "kb", GAUSS: "gauss"}


@pytest.fixture(scope="module")
def lib():
    return binding.load_library()


def c_bound(lib, B, window, q, sigma):
    b = ctypes.c_double(-1.0)
    assert lib.sgl_nfft_error_bound(B, window, q, ctypes.c_double(sigma), ctypes.byref(b)) == 0
    return b.value


@pytest.mark.parametrize("B,window,q,sigma", [(4, KB, 2, 2.0), (8, KB, 4, 2.0), (6, GAUSS, 3, 2.0),
                                              (5, KB, 3, 1.5), (8, GAUSS, 6, 2.5), (12, KB, 5, 3.0)])
def test_bound_equals_the_oracles_definition(lib, B, window, q, sigma):
    ref = nfft.sgl_nfft_bound(B, q, sigma, NAMES[window])
    assert c_bound(lib, B, window, q, sigma) == pytest.approx(ref, rel=1e-6)


@pytest.mark.parametrize("B", [4, 8])
def test_bound_reaches_rounding_level_at_large_cutoff(lib, B):
    # KB at q = 8: both sides see only rounding (the window error is below 1e-13)
    assert c_bound(lib, B, KB, 8, 2.0) <= 1e-12
    assert nfft.sgl_nfft_bound(B, 8, 2.0, "kb") <= 1e-12


@pytest.mark.parametrize("sigma", [2.0, 3.0])
@pytest.mark.parametrize("q", [2, 4, 6, 8, 10])
def test_gaussian_bound_below_the_papers_closed_form(lib, q, sigma):
    # the theorem bounds the error of every coefficient vector by C ||w||_1, with C in closed form
    assert c_bound(lib, 8, GAUSS, q, sigma) <= nfft.gauss_error_bound(3, sigma, q)


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "gauss_nfft_error_constant.json")


@pytest.mark.parametrize("case", json.load(open(GOLDEN))["cases"], ids=lambda c: "d%d-s%g-q%d" % (c["d"], c["sigma"], c["q"]))
def test_gaussian_closed_form_equals_the_theorems_constant(case):
    # the closed form of the theorem on the d-dimensional NFFT error, evaluated by hand (golden file)
    assert nfft.gauss_error_bound(case["d"], case["sigma"], case["q"]) == pytest.approx(case["C"], rel=1e-13)


@pytest.mark.parametrize("d,sigma", [(1, 2.0), (2, 2.0), (3, 2.0), (3, 3.0)])
def test_gaussian_closed_form_decay_rate_and_prefactor_limit(d, sigma):
    # large q: the prefactor tends to (2^d - 1) 2^d and the ratio of consecutive cutoffs to
    # e^{-pi E}, E = 1 - (1 + d / (2 sigma - 1)) / (2 sigma) -- the exponent and the constant
    # pinned separately from the golden values
    E = 1.0 - (1.0 + d / (2.0 * sigma - 1.0)) / (2.0 * sigma)
    q = 200
    ratio = nfft.gauss_error_bound(d, sigma, q + 1) / nfft.gauss_error_bound(d, sigma, q)
    assert math.log(ratio) == pytest.approx(-math.pi * E, abs=2e-4)
    pref = nfft.gauss_error_bound(d, sigma, q) * math.exp(q * math.pi * E)
    # corrections at finite q: (1 + 1/(2 pi q))^d - 1 from the first term, O(q^{-d/2}) from the second
    tol = 1.2 * d / (2 * math.pi * q) + 1.5 * (3 ** d - 1) / ((2 ** d - 1) * 2 ** d) * q ** (-d / 2)
    assert pref == pytest.approx((2 ** d - 1) * 2 ** d, rel=tol)


def test_gaussian_closed_form_rejects_small_oversampling():
    with pytest.raises(ValueError):
        nfft.gauss_error_bound(3, 1.3, 8)


def test_bound_holds_for_the_oracle_nfft():
    # a random trigonometric polynomial on the grid sizes of the oracle's NFFT, measured error
    # against the direct sum: below bound * ||omega||_1 (bound from the same single-frequency errors)
    rng = np.random.default_rng(5)
    n, sigma = (8, 6, 6), 2.0
    for window, q in (("kb", 3), ("gauss", 4), ("kb", 5)):
        om = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        t = rng.uniform(0, 2 * math.pi, (300, 3))
        approx = nfft.nfft(om, t, sigma, q, window)
        ks = [np.arange(nj) - nj // 2 for nj in n]
        exact = np.einsum("abc,ia,ib,ic->i", om, np.exp(1j * t[:, :1] * ks[0]), np.exp(1j * t[:, 1:2] * ks[1]),
                          np.exp(1j * t[:, 2:] * ks[2]))
        b = 1.0
        for d in range(3):
            b *= 1.0 + nfft.single_frequency_error(int(round(sigma * n[d])), n[d], n[d] // 2, q, window)
        assert np.abs(approx - exact).max() <= (b - 1.0) * np.abs(om).sum()


def test_bound_decreases_with_the_cutoff_and_kb_beats_gauss(lib):
    kb = [c_bound(lib, 16, KB, q, 2.0) for q in range(2, 8)]
    ga = [c_bound(lib, 16, GAUSS, q, 2.0) for q in range(2, 8)]
    assert all(b < a for a, b in zip(kb, kb[1:]))
    assert all(b < a for a, b in zip(ga, ga[1:]))
    assert all(k < g for k, g in zip(kb, ga))


@pytest.mark.parametrize("tol", [1e-3, 1e-6, 1e-9, 1e-12])
def test_choose_cutoff_is_the_smallest_sufficient_q(lib, tol):
    q = ctypes.c_int(0)
    assert lib.sgl_choose_cutoff(32, KB, ctypes.c_double(2.0), ctypes.c_double(tol), ctypes.byref(q)) == 0
    assert c_bound(lib, 32, KB, q.value, 2.0) <= tol
    if q.value > 1:
        assert c_bound(lib, 32, KB, q.value - 1, 2.0) > tol


def test_argument_errors(lib):
    b, q = ctypes.c_double(), ctypes.c_int()
    assert lib.sgl_nfft_error_bound(0, KB, 4, ctypes.c_double(2.0), ctypes.byref(b)) == 1
    assert lib.sgl_nfft_error_bound(8, 7, 4, ctypes.c_double(2.0), ctypes.byref(b)) == 1
    assert lib.sgl_nfft_error_bound(8, KB, 17, ctypes.c_double(2.0), ctypes.byref(b)) == 1
    assert lib.sgl_choose_cutoff(8, KB, ctypes.c_double(2.0), ctypes.c_double(0.0), ctypes.byref(q)) == 1
    assert lib.sgl_choose_cutoff(8, GAUSS, ctypes.c_double(2.0), ctypes.c_double(1e-300), ctypes.byref(q)) == 6


def test_bound_is_attained_by_the_worst_single_frequency():
    # not vacuous: over the single coefficient vectors e_k (k on axis 0, 0 on the others), the
    # oracle's 3-D NFFT at many points shows an error of at least half of axis 0's term of the
    # bound (the axes at k = 0 add next to nothing), and never more than the whole bound
    n, sigma, q, window = (8, 6, 6), 2.0, 3, "kb"
    e0 = nfft.single_frequency_error(int(round(sigma * n[0])), n[0], n[0] // 2, q, window)
    t = np.random.default_rng(9).uniform(0, 2 * math.pi, (4000, 3))
    om = np.zeros(n, complex)
    worst = 0.0
    for k in range(-(n[0] // 2), n[0] // 2):
        om[:] = 0
        om[k + n[0] // 2, n[1] // 2, n[2] // 2] = 1.0
        worst = max(worst, float(np.abs(nfft.nfft(om, t, sigma, q, window) - np.exp(1j * k * t[:, 0])).max()))
    b = 1.0
    for d in range(3):
        b *= 1.0 + nfft.single_frequency_error(int(round(sigma * n[d])), n[d], n[d] // 2, q, window)
    assert 0.5 * e0 <= worst <= b - 1.0


# ---- error-driven choice of (sigma, q) with the GB300 cost model (host code)
SIGMAS = (1.5, 2.0, 2.5, 3.0, 4.0)
TAP_MS = {0: (9.3 + 15.9) / 4.096e9, 1: (0.89 + 1.49) / 4.096e9}
CELL_MS = {0: 3.81 / (273 * 145 * 256), 1: 0.69 / (273 * 145 * 256)}


def model_ms(B, M, prec, sigma, q):
    cells = 1.0
    for d, n in enumerate((4 * B, 2 * B, 2 * B)):
        N = nfft.fft_size(sigma * n)
        cells *= N // 2 + 2 * q + 1 if d < 2 and N // 2 + 2 * q + 1 <= N else N
    return M * (2 * q) ** 3 * TAP_MS[prec] + cells * CELL_MS[prec]


def choose(lib, B, M, prec, tol, window=KB):
    sg, q, ms = ctypes.c_double(), ctypes.c_int(), ctypes.c_double()
    st = lib.sgl_choose_params(B, M, prec, window, ctypes.c_double(tol), ctypes.byref(sg), ctypes.byref(q), ctypes.byref(ms))
    return st, sg.value, q.value, ms.value


@pytest.mark.parametrize("B,M,prec,tol", [(16, 10**4, 1, 1e-6), (32, 10**6, 1, 1e-6), (32, 10**6, 0, 1e-12),
                                          (64, 10**3, 0, 1e-9), (64, 10**7, 1, 1e-4), (8, 0, 0, 1e-10)])
def test_choose_params_meets_tol_at_the_cheapest_modelled_pair(lib, B, M, prec, tol):
    st, sg, q, ms = choose(lib, B, M, prec, tol)
    assert st == 0
    assert c_bound(lib, B, KB, q, sg) <= tol
    if q > 1:
        assert c_bound(lib, B, KB, q - 1, sg) > tol          # smallest q for that sigma
    assert ms == pytest.approx(model_ms(B, M, prec, sg, q), rel=1e-9)
    # no other candidate sigma reaches tol more cheaply (each at its own smallest q)
    for s2 in SIGMAS:
        for q2 in range(1, 17):
            if c_bound(lib, B, KB, q2, s2) <= tol:
                assert model_ms(B, M, prec, s2, q2) >= ms * (1 - 1e-12)
                break


def test_choose_params_trades_grid_for_taps(lib):
    # many points make taps dear (a larger sigma with a smaller q wins); few points make the grid dear
    _, sg_many, q_many, _ = choose(lib, 32, 10**8, 1, 1e-7)
    _, sg_few, q_few, _ = choose(lib, 32, 10**2, 1, 1e-7)
    assert sg_many > sg_few and q_many < q_few


def test_choose_params_argument_errors(lib):
    sg, q = ctypes.c_double(), ctypes.c_int()
    assert lib.sgl_choose_params(0, 10, 0, KB, ctypes.c_double(1e-6), ctypes.byref(sg), ctypes.byref(q), None) == 1
    assert lib.sgl_choose_params(8, -1, 0, KB, ctypes.c_double(1e-6), ctypes.byref(sg), ctypes.byref(q), None) == 1
    assert lib.sgl_choose_params(8, 10, 0, KB, ctypes.c_double(0.0), ctypes.byref(sg), ctypes.byref(q), None) == 1
    assert lib.sgl_choose_params(8, 10, 0, KB, ctypes.c_double(1e-40), ctypes.byref(sg), ctypes.byref(q), None) == 6
