"""The symmetry-reduced FFT passes against the whole-grid passes and against the oracle (marked gpu).

eta is even in kappa0 and has the parity of m in kappa1 (Sect. 6), so the oversampled grid of the
NFFT (Sect. 2) is even in l0 and alpha(l0, -l1, l2) = alpha(l0, l1, l2 + N2/2).  By default the
FFT passes transform the radial lines kappa1 >= 0 and the angular lines of
[0, N0/2] x [0, N1/2] only, and fill the q halo rows on each side of both windowed axes by
mirroring; the adjoint folds in the same places (in both the register and the generic FFT
kernels).  SGL_FLAG_FULL_GRID transforms every kept line.
Both compute the same operator, so they agree to rounding.

Points at the origin (t0 = pi), at the largest radius (t0 = 0) and on both poles (theta = 0, pi)
put taps on every halo row.  The bounds are a few times the measured differences (`envelope`).
"""
import numpy as np
import pytest
import torch

import paper_1809_10786_gb300 as sgl
from envelope import check
from paper_1809_10786_gb300 import inputs
from oracle import direct

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def edge_points(M, seed):
    """Seeded Gaussian points plus points on the boundary rows of both windowed axes."""
    x = inputs.points_gaussian(M, seed)
    r = 0.9 * np.sqrt((x ** 2).sum(1)).max()
    extra = [[0.0, 0.0, 0.0], [0.0, 0.0, 0.3], [0.0, 0.0, -0.3], [0.0, 0.0, r], [0.0, 0.0, -r],
             [r, 0.0, 0.0], [0.0, -r, 1e-9], [1e-3, 0.0, 0.0], [0.0, 1e-3, -1e-3], [2.0, 1e-7, 1e-7]]
    return np.concatenate([x, np.array(extra)], 0)


def regular(x):
    """Points where the chain rule is well conditioned (the gradient's singular places r = 0,
    r = rho and sin theta = 0 set the singular terms to zero instead of their limits)."""
    r = np.sqrt((x ** 2).sum(1))
    rho = r.max()
    with np.errstate(invalid="ignore", divide="ignore"):
        st = np.sqrt(x[:, 0] ** 2 + x[:, 1] ** 2) / r
    return (r >= 0.05 * rho) & (r <= 0.95 * rho) & (st > 0.1)


def run(B, x, prec, full, seed, **kw):
    M = len(x)
    c = inputs.coefficients(B, seed)
    y = inputs.values(M, seed + 1)
    g = inputs.complex_normal(M, seed + 2)
    p = sgl.Plan(B, M, precision=prec, q=8, device=DEV, full_grid=full, **kw)
    p.set_points(gpu(x))
    f, gx = p.forward_grad(gpu(c), gpu(g))
    a = p.adjoint(gpu(y))
    out = f.cpu().numpy(), gx.cpu().numpy(), a.cpu().numpy()
    p.close()
    return out, (c, y, g)


# FP64 with double-float windowed loops (default) or binary64 ones, FP32-mixed with the tensor-core
# interpolation (default at q = 8) or the CUDA-core kernels
CONFIGS = [("fp64", sgl.PREC_FP64, {}, 2e-12), ("fp64-native", sgl.PREC_FP64, {"native_fp64": True}, 1e-13),
           ("fp32-tc", sgl.PREC_FP32_MIXED, {}, 2e-6), ("fp32-simt", sgl.PREC_FP32_MIXED, {"simt": True}, 2e-6)]


# B = 20, 24: lengths 160 / 80 and 192 / 96, which take the generic FFT kernel
@pytest.mark.parametrize("B", [16, 20, 24, 32, 64])
@pytest.mark.parametrize("name,prec,kw,tol", CONFIGS)
def test_reduced_grid_matches_full_grid(B, name, prec, kw, tol):
    x = edge_points(2000, 9700 + B)
    (f_h, g_h, a_h), _ = run(B, x, prec, False, 9710 + B, **kw)
    (f_f, g_f, a_f), _ = run(B, x, prec, True, 9710 + B, **kw)
    check("half grid vs full forward B=%d %s" % (B, name), rel(f_h, f_f), tol)
    check("half grid vs full adjoint B=%d %s" % (B, name), rel(a_h, a_f), tol)
    # every point, the singular places included (both set the same terms to zero)
    check("half grid vs full gradient B=%d %s" % (B, name), rel(g_h, g_f), 10 * tol)


@pytest.mark.parametrize("B,prec,tol_f,tol_a,tol_g", [(24, sgl.PREC_FP64, 1e-10, 1e-10, 1e-9),
                                                      (32, sgl.PREC_FP64, 1e-10, 1e-10, 1e-9),
                                                      (32, sgl.PREC_FP32_MIXED, 3e-6, 3e-6, 3e-5)])
def test_reduced_grid_against_the_oracle(B, prec, tol_f, tol_a, tol_g):
    # B = 24: grid lengths 192 and 96 take the generic FFT kernel
    x = edge_points(300, 9800 + B)
    (f, gx, a), (c, y, g) = run(B, x, prec, False, 9810 + B)
    f_ref, _ = direct.forward(B, x, c)
    a_ref, _ = direct.adjoint(B, x, y)
    ok = regular(x)
    g_ref, _ = direct.grad_points(B, x[ok], c, g[ok])
    check("half grid oracle forward B=%d prec=%d" % (B, prec), rel(f, f_ref), tol_f)
    check("half grid oracle adjoint B=%d prec=%d" % (B, prec), rel(a, a_ref), tol_a)
    check("half grid oracle gradient B=%d prec=%d" % (B, prec), rel(gx[ok], g_ref), tol_g)
    assert np.all(np.isfinite(gx))


def test_reduced_grid_adjoint_identity():
    # <Lambda c, y> = <c, Lambda^H y> for the reduced pair (exact adjoints of one operator)
    B = 32
    x = edge_points(1500, 9900)
    (f, _, a), (c, y, _) = run(B, x, sgl.PREC_FP64, False, 9910)
    lhs = np.vdot(y, f)
    rhs = np.vdot(a, c)
    assert abs(lhs - rhs) <= 1e-12 * np.abs(y).sum() * np.abs(f).max()


@pytest.mark.parametrize("B,kw,expect", [(32, {}, True), (32, {"full_grid": True}, False), (32, {"generic_fft": True}, True),
                                         (8, {}, False), (24, {}, True)])
def test_plan_reports_where_the_reduced_grid_applies(B, kw, expect):
    # B = 8: axis 1 is periodic at q = 8
    p = sgl.Plan(B, 10, precision=sgl.PREC_FP32_MIXED, q=8, device=DEV, **kw)
    assert p.info()["sym_grid"] is expect
