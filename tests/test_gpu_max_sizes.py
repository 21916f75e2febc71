"""The largest plans the library accepts, against the oracle (marked gpu).

B = 128 is the largest bandwidth (grid lengths 1024 x 512 x 512 at sigma = 2, the longest the
register FFT kernels take; Nc = 707,264 coefficients); q = 16 the widest window (32 taps per
axis: the CUDA-core kernels with one 32-lane group per point).  The oracle is the direct sum on
a small point sample; the FP64 bound is the metric's 1e-10, the FP32 ones a few times the
measured errors (`envelope`).
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


def regular(x):
    # away from the gradient's singular places (r = 0, r = rho, sin theta = 0)
    r = np.sqrt((x ** 2).sum(1))
    st = np.sqrt(x[:, 0] ** 2 + x[:, 1] ** 2) / np.maximum(r, 1e-300)
    return (r >= 0.05 * r.max()) & (r <= 0.95 * r.max()) & (st > 0.1)


# measured on GB300: FP64 1.7e-14 / 2.0e-14 / 1.6e-13, FP32 1.7e-7 / 8.1e-8 / 4.4e-7
@pytest.mark.parametrize("prec,tol_f,tol_a,tol_g", [(sgl.PREC_FP64, 1e-10, 1e-10, 1e-9),
                                                    (sgl.PREC_FP32_MIXED, 1e-6, 5e-7, 3e-6)])
def test_bandwidth_128(prec, tol_f, tol_a, tol_g):
    B, M = 128, 120
    c = inputs.coefficients(B, 9900)
    x = inputs.points_gaussian(M, 9901)
    y = inputs.values(M, 9902)
    g = inputs.complex_normal(M, 9903)
    p = sgl.Plan(B, M, precision=prec, q=8, device=DEV)
    assert p.info()["N"] == [1024, 512, 512] and p.info()["sym_grid"]
    p.set_points(gpu(x))
    f, gx = p.forward_grad(gpu(c), gpu(g))
    a = p.adjoint(gpu(y)).cpu().numpy()
    f, gx = f.cpu().numpy(), gx.cpu().numpy()
    f_ref, _ = direct.forward(B, x, c)
    a_ref, _ = direct.adjoint(B, x, y)
    ok = regular(x)
    # the binary64 oracle's gradient divides factorials that overflow once l + m > 170 (its
    # P_{l, m +- 1} ratios); its long-double build covers B = 128
    g_ref, _ = direct.grad_points(B, x[ok], c, g[ok], kind="long double")
    check("B=128 forward prec=%d" % prec, rel(f, f_ref), tol_f)
    check("B=128 adjoint prec=%d" % prec, rel(a, a_ref), tol_a)
    check("B=128 gradient prec=%d" % prec, rel(gx[ok], g_ref), tol_g)


# FP32: measured forward 4.7e-6, adjoint 8.5e-6 (a 32-lane group sums 32^3 taps per point in
# binary32, and spreading adds them to the grid one tap at a time)
@pytest.mark.parametrize("prec,win,tol", [(sgl.PREC_FP64, sgl.WIN_KB, 1e-10), (sgl.PREC_FP64, sgl.WIN_GAUSS, 1e-10),
                                          (sgl.PREC_FP32_MIXED, sgl.WIN_KB, 2e-5)])
def test_cutoff_16(prec, win, tol):
    B, M = 20, 1500
    c = inputs.coefficients(B, 9910)
    x = inputs.points_gaussian(M, 9911)
    y = inputs.values(M, 9912)
    p = sgl.Plan(B, M, precision=prec, window=win, q=16, device=DEV)
    p.set_points(gpu(x))
    f = p.forward(gpu(c)).cpu().numpy()
    a = p.adjoint(gpu(y)).cpu().numpy()
    f_ref, _ = direct.forward(B, x, c)
    a_ref, _ = direct.adjoint(B, x, y)
    check("q=16 forward prec=%d win=%d" % (prec, win), rel(f, f_ref), tol)
    check("q=16 adjoint prec=%d win=%d" % (prec, win), rel(a, a_ref), tol)
