"""Inverse transform (iNFSGLFT) on the GPU against the oracle's dense CGNR / CGNE (marked gpu).

The GPU runs the same iterations with the fast transform pair in place of the dense matrix.
Intermediate CG iterates are not a stable function of the operator: on the B = 5, M = 500
system below a 1e-14 relative perturbation of Lambda moves the 30th CGNR iterate by ~1e-4, and
perturbing the forward and the adjoint matrices independently by 1e-14 (a pair that is no
longer exactly adjoint, as two rounded fast transforms are not) moves the residual norms of
iterations 10-30 by 0.4-11 % (1e-15: by 1e-4).  So the pins are the early residuals (iteration
5), the size of the later ones, and the least-squares / minimum-norm solutions reached at
convergence.
"""
import numpy as np
import pytest
import torch

import paper_1809_10786_gb300 as sgl
from paper_1809_10786_gb300 import inputs
from oracle import direct, inverse

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def plan(B, x, prec=sgl.PREC_FP64, q=8, native=False):
    p = sgl.Plan(B, len(x), precision=prec, q=q, device=DEV, native_fp64=native)
    p.set_points(gpu(x))
    return p


# later residuals: within 2 % of the oracle's with the binary64 windowed loops (transform errors
# ~1e-15, the sensitivity above at 1e-15 is ~1e-4), 25 % with the double-float loops (errors of
# order 1e-14, the sensitivity above at 1e-14 reaches 11 %)
@pytest.mark.parametrize("native,later", [(True, 0.02), (False, 0.25)])
def test_cgnr_follows_the_oracle_and_reaches_least_squares(native, later):
    B, M = 5, 500                                  # Nc = 55, cond(Lambda) ~ 150
    x = inputs.points_gaussian(M, 9305)
    L = inverse.matrix(B, x)
    f = L @ inputs.coefficients(B, 9306) + 1e-3 * inputs.complex_normal(M, 9307)
    p = plan(B, x, native=native)
    _, res_or = inverse.cgnr(L, f, np.zeros(L.shape[1], complex), 30)
    gpu_res = []
    for it in (5, 10, 20, 30):
        _, r, k = p.inverse(gpu(f), iters=it, method="cgnr")
        assert k == it
        gpu_res.append(r)
        # early residual norms follow the oracle's closely, later ones to the sensitivity above
        assert r == pytest.approx(res_or[it] / res_or[0], rel=1e-6 if it == 5 else later)
    assert all(b <= a * (1 + 1e-3) for a, b in zip(gpu_res, gpu_res[1:]))
    c, res, k = p.inverse(gpu(f), iters=300, tol=0.0, method="cgnr")
    c_ls = np.linalg.lstsq(L, f, rcond=None)[0]
    assert rel(c.cpu().numpy(), c_ls) <= 1e-8
    assert res == pytest.approx(np.linalg.norm(f - L @ c_ls) / np.linalg.norm(f), rel=1e-6)


def test_cgne_reaches_minimum_norm_solution():
    B, M = 6, 40                                   # Nc = 91 > M: automatic choice is CGNE
    x = inputs.points_gaussian(M, 9316)
    L = inverse.matrix(B, x)
    f = inputs.complex_normal(M, 9317)
    p = plan(B, x)
    c, res, k = p.inverse(gpu(f), iters=400, tol=1e-13)
    c_mn = np.linalg.lstsq(L, f, rcond=None)[0]
    assert res <= 1e-12
    assert k < 400
    assert rel(c.cpu().numpy(), c_mn) <= 1e-7


def test_tolerance_stops_early_and_initial_guess_is_used():
    B, M = 5, 500
    x = inputs.points_gaussian(M, 9305)
    c_true = inputs.coefficients(B, 9326)
    f, _ = direct.forward(B, x, c_true)
    p = plan(B, x)
    c, res, k = p.inverse(gpu(f), iters=500, tol=1e-9)
    assert res <= 1e-9 and k < 500
    assert rel(c.cpu().numpy(), c_true) <= 1e-6
    # starting from the solution: no iteration is needed
    c2, res2, k2 = p.inverse(gpu(f), coef0=gpu(c_true), iters=50, tol=1e-9)
    assert k2 == 0 and res2 <= 1e-9


def test_midpoint_guess_matches_the_oracle():
    B, N, kappa = 4, 16, 5.0
    x = inverse.cartesian_grid(N, kappa)
    f, _ = direct.forward(B, x, inputs.coefficients(B, 9336))
    w = (2.0 * kappa / N) ** 3 * np.exp(-np.sum(x * x, axis=1))
    p = plan(B, x)
    g = p.midpoint_guess(gpu(f), gpu(w)).cpu().numpy()
    assert rel(g, inverse.midpoint_guess(B, x, f, kappa, N)) <= 1e-10


@pytest.mark.parametrize("native", [True, False])
def test_paper_last_test_setup_small(native):
    # Sect. 8, last test, at a size the dense oracle handles: Cartesian grid G_N, kappa = 5,
    # exact samples of random coefficients, CGNR from the mid-point rule
    B, N, kappa = 4, 14, 5.0
    x = inverse.cartesian_grid(N, kappa)
    c_true = inputs.coefficients(B, 9346)
    f, _ = direct.forward(B, x, c_true)
    w = (2.0 * kappa / N) ** 3 * np.exp(-np.sum(x * x, axis=1))
    p = plan(B, x, native=native)
    c0 = p.midpoint_guess(gpu(f), gpu(w))
    L = inverse.matrix(B, x)
    c_or, res_or = inverse.cgnr(L, f, c0.cpu().numpy(), 40)
    nf = np.linalg.norm(f)
    # Nc = 30 unknowns: in exact arithmetic CGNR ends by iteration 30, and past it the residual is
    # set by rounding (the oracle alone gave 8.9e-9 and 5.5e-9 at iteration 40 from initial
    # guesses 1e-16 apart).  Iterations 10, 16 and 20 move by up to 26 %, 38 % and 64 % under
    # independent 1e-13 perturbations of the forward and adjoint matrices (the size of the
    # double-float transforms' rounding), iteration 15 by 2.6e-8 (1.5e-5 under 1e-12; 16 seeds
    # each), so iteration 15 carries the pin; iteration 40 only its size.
    c, res, k = p.inverse(gpu(f), coef0=c0, iters=15, method="cgnr")
    assert res == pytest.approx(res_or[15] / nf, rel=1e-3)
    c, res, k = p.inverse(gpu(f), coef0=c0, iters=40, method="cgnr")
    assert res <= res_or[0] / nf
    assert res <= 10.0 * res_or[40] / nf
    # run to convergence: the consistent system gives back the coefficients
    c, res, k = p.inverse(gpu(f), coef0=c0, iters=2000, tol=1e-10, method="cgnr")
    assert res <= 1e-10
    assert rel(c.cpu().numpy(), c_true) <= 1e-6


def test_paper_last_test_b8_reaches_small_error_like_the_oracle():
    # Sect. 8, last test, B = 8, kappa = 5, N = 25 (M = 15625): the paper reports a small error
    # after many iterations.  Lambda has condition ~1.7e8 here; the dense-oracle CGNR reaches
    # max abs / rel error 7.3e-5 / 2.1e-4 after 1000 iterations (from 1.7e-2 / 5.4e-2), and the
    # GPU's run with the fast transform pair follows it to within cond * (its NFFT error).
    B, N, kappa = 8, 25, 5.0
    x = inverse.cartesian_grid(N, kappa)
    c_true = inputs.coefficients(B, 9401)
    L = inverse.matrix(B, x)
    f = L @ c_true
    w = (2.0 * kappa / N) ** 3 * np.exp(-np.sum(x * x, axis=1))
    c_or, _ = inverse.cgnr(L, f, inverse.midpoint_guess(B, x, f, kappa, N), 1000)
    p = plan(B, x)
    c0 = p.midpoint_guess(gpu(f), gpu(w))
    c, res, k = p.inverse(gpu(f), coef0=c0, iters=1000, method="cgnr")
    assert k == 1000 and res <= 1e-8

    def errs(c):
        d = np.abs(c - c_true)
        return d.max(), (d / np.abs(c_true)).max()
    a0, r0 = errs(c0.cpu().numpy())
    a, r = errs(c.cpu().numpy())
    a_or, r_or = errs(c_or)
    assert a <= 0.02 * a0 and r <= 0.02 * r0
    assert a <= 2 * a_or and r <= 2 * r_or


def test_fp32_mixed_plan_converges_to_its_precision():
    B, M = 5, 500
    x = inputs.points_gaussian(M, 9305)
    L = inverse.matrix(B, x)
    f = L @ inputs.coefficients(B, 9356)
    p = plan(B, x, prec=sgl.PREC_FP32_MIXED)
    c, res, k = p.inverse(gpu(f), iters=200)
    c_ls = np.linalg.lstsq(L, f, rcond=None)[0]
    assert res <= 1e-5
    assert rel(c.cpu().numpy(), c_ls) <= 1e-3


def test_inverse_argument_errors():
    p = sgl.Plan(4, 10, device=DEV)
    with pytest.raises(sgl.SGLError):
        p.inverse(torch.zeros(0, dtype=torch.complex128, device=DEV))      # no points set yet
    p.set_points(gpu(inputs.points_gaussian(10, 9366)))
    lib = p.lib
    v = torch.zeros(10, dtype=torch.complex128, device=DEV)
    c = torch.zeros(p.Nc, dtype=torch.complex128, device=DEV)
    import ctypes
    assert lib.sgl_inverse(p._h, ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(c.data_ptr()), 5, 0.0, 3, None, None) == 1
    assert lib.sgl_inverse(p._h, ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(c.data_ptr()), -1, 0.0, 0, None, None) == 1
