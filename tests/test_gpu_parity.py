"""GPU parity of the C-ABI path against the CPU oracle (marked gpu).

Tolerances: FP64 path <= 1e-10 max-abs-error / max-abs-value at window cutoff q = 8
(Kaiser-Bessel, sigma = 2); the FP32-mixed path is bounded by a measured envelope.
The exported trigonometric coefficients are exact (the factorization is exact, Sect. 7),
so they match the oracle's factorization to rounding.  The GPU forward/adjoint pair
is an exact adjoint pair of the same approximate operator, so the adjoint identity
holds to rounding.
"""
import numpy as np
import pytest
import torch

import paper_1809_10786_gb300 as sgl
from envelope import check
from paper_1809_10786_gb300 import inputs
from oracle import direct, factorization as fz

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def case(B, M, seed):
    c = inputs.coefficients(B, seed)
    x = inputs.points_gaussian(M, seed + 1)
    y = inputs.values(M, seed + 2)
    return c, x, y


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def plan_for(B, M, prec=sgl.PREC_FP64, win=sgl.WIN_KB, q=8, sigma=2.0, x=None, **kw):
    p = sgl.Plan(B, M, precision=prec, window=win, q=q, sigma=sigma, **kw)
    if x is not None:
        p.set_points(gpu(x))
    return p


@pytest.mark.parametrize("B,M", [(1, 10), (2, 40), (8, 1000), (13, 300), (21, 500)])
def test_trig_coeffs_equal_oracle_factorization(B, M):
    c, x, _ = case(B, M, 1000 + B)
    p = plan_for(B, M, q=min(8, B), x=x)          # eta does not depend on the window; small grids need small q
    eta = p.trig_coeffs(gpu(c)).cpu().numpy()
    ref = fz.eta(B, c, p.rho())
    K0, K1 = 2 * B - 2, B - 1
    ref = ref[2 * B - K0:2 * B + K0 + 1, 2 * B - K1:2 * B + K1 + 1, 2 * B - K1:2 * B + K1 + 1]
    assert rel(eta, ref) <= 1e-13


@pytest.mark.parametrize("native", [False, True])
@pytest.mark.parametrize("B,M,win,q", [(8, 1000, sgl.WIN_KB, 8), (13, 700, sgl.WIN_KB, 8), (20, 3333, sgl.WIN_KB, 8),
                                       (8, 500, sgl.WIN_GAUSS, 12), (4, 257, sgl.WIN_KB, 7)])
def test_forward_and_adjoint_fp64(B, M, win, q, native):
    # native: binary64 hot loops; otherwise double-float (the FP64 plan's default)
    c, x, y = case(B, M, 2000 + B)
    p = plan_for(B, M, win=win, q=q, x=x, native_fp64=native)
    f = p.forward(gpu(c)).cpu().numpy()
    a = p.adjoint(gpu(y)).cpu().numpy()
    f_ref, _ = direct.forward(B, x, c)
    a_ref, _ = direct.adjoint(B, x, y)
    assert rel(f, f_ref) <= 1e-10
    assert rel(a, a_ref) <= 1e-10


@pytest.mark.parametrize("prec,tol", [(sgl.PREC_FP64, 1e-13), (sgl.PREC_FP32_MIXED, 2e-8)])   # FP32: measured 4.4e-9
def test_adjoint_identity(prec, tol):
    B, M = 16, 4000
    c, x, y = case(B, M, 3000)
    p = plan_for(B, M, prec=prec, x=x)
    f = p.forward(gpu(c)).cpu().numpy()
    a = p.adjoint(gpu(y)).cpu().numpy()
    lhs, rhs = np.vdot(y, f), np.vdot(a, c)
    check("adjoint identity B=16 prec=%d" % prec, abs(lhs - rhs) / (np.linalg.norm(f) * np.linalg.norm(y)), tol)


# about 5x the measured forward / adjoint errors: q = 4: 1.7e-7 / 1.1e-7; q = 6: 3.3e-7 / 1.0e-7;
# q = 8: 5.6e-7 / 9.4e-8
@pytest.mark.parametrize("q,bound_f,bound_a", [(4, 1e-6, 6e-7), (6, 1.7e-6, 5e-7), (8, 3e-6, 5e-7)])
def test_fp32_mixed_error_envelope(q, bound_f, bound_a):
    B, M = 16, 3000
    c, x, y = case(B, M, 4000 + q)
    p = plan_for(B, M, prec=sgl.PREC_FP32_MIXED, q=q, x=x)
    f = p.forward(gpu(c)).cpu().numpy()
    a = p.adjoint(gpu(y)).cpu().numpy()
    f_ref, _ = direct.forward(B, x, c)
    a_ref, _ = direct.adjoint(B, x, y)
    check("fp32 envelope B=16 q=%d forward" % q, rel(f, f_ref), bound_f)
    check("fp32 envelope B=16 q=%d adjoint" % q, rel(a, a_ref), bound_a)


@pytest.mark.parametrize("prec,tol,native", [(sgl.PREC_FP64, 1e-9, False), (sgl.PREC_FP64, 1e-9, True),
                                             (sgl.PREC_FP32_MIXED, 1e-4, False)])     # FP32: measured 1.8e-5
def test_grad_points_against_oracle(prec, tol, native):
    B, M = 12, 1500
    c, x, g = case(B, M, 5000)
    p = plan_for(B, M, prec=prec, x=x, native_fp64=native)
    gx = p.grad_points(gpu(c), gpu(g)).cpu().numpy()
    ref, _ = direct.grad_points(B, x, c, g)
    check("gradient B=12 prec=%d native=%d" % (prec, native), rel(gx, ref), tol)


def test_grad_points_against_gpu_finite_differences():
    # the gradient is the derivative of the GPU forward map itself (rho held fixed)
    B, M = 8, 64
    c, x, g = case(B, M, 6000)
    p = plan_for(B, M, x=x)
    gx = p.grad_points(gpu(c), gpu(g)).cpu().numpy()
    rho = p.rho()
    # keep rho fixed: add a far anchor point that fixes max |x|
    anchor = np.array([[0.0, 0.0, rho / (1 + 2.0 ** -20)]])
    h = 1e-6
    fd = np.zeros((M, 3))
    q = plan_for(B, M + 1)
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        q.set_points(gpu(np.vstack([x + e, anchor])))
        fp = q.forward(gpu(c)).cpu().numpy()[:M]
        q.set_points(gpu(np.vstack([x - e, anchor])))
        fm = q.forward(gpu(c)).cpu().numpy()[:M]
        fd[:, d] = np.real(np.conj(g) * (fp - fm) / (2 * h))
    inner = np.linalg.norm(x, axis=1) < rho * 0.999
    assert np.abs(gx[inner] - fd[inner]).max() <= 1e-6 * np.abs(fd).max()


def test_empty_and_single_point():
    B = 6
    c, x, y = case(B, 1, 7000)
    p = plan_for(B, 5)
    p.set_points(gpu(np.zeros((0, 3))))
    assert p.forward(gpu(c)).numel() == 0
    a = p.adjoint(torch.zeros(0, dtype=torch.complex128, device=DEV)).cpu().numpy()
    assert np.all(a == 0)
    p.set_points(gpu(x))
    f = p.forward(gpu(c)).cpu().numpy()
    f_ref, _ = direct.forward(B, x, c)
    assert rel(f, f_ref) <= 1e-10


def test_degenerate_points():
    # origin, the z-axis (both poles), a repeated point and the maximum radius
    B = 9
    c = inputs.coefficients(B, 7100)
    x = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 1.3], [0.0, 0.0, -0.7], [0.4, -0.2, 0.1], [0.4, -0.2, 0.1],
                  [2.5, 0.0, 0.0], [-1e-12, 0.0, 0.5]])
    y = inputs.values(len(x), 7101)
    p = plan_for(B, len(x), x=x)
    f = p.forward(gpu(c)).cpu().numpy()
    a = p.adjoint(gpu(y)).cpu().numpy()
    f_ref, _ = direct.forward(B, x, c)
    a_ref, _ = direct.adjoint(B, x, y)
    assert rel(f, f_ref) <= 1e-10
    assert rel(a, a_ref) <= 1e-10
    assert np.all(np.isfinite(p.grad_points(gpu(c), gpu(y)).cpu().numpy()))


def test_nonfinite_point_is_reported():
    B = 4
    x = inputs.points_gaussian(10, 7200)
    x[3, 1] = np.nan
    p = plan_for(B, 10, x=x)
    with pytest.raises(sgl.SGLError) as ei:
        p.sync()
    assert ei.value.status == 4
    p.sync()                          # flag cleared


def test_state_and_argument_errors():
    p = plan_for(4, 10)
    c = gpu(inputs.coefficients(4, 1))
    with pytest.raises(sgl.SGLError) as ei:
        p.forward(c)
    assert ei.value.status == 7
    with pytest.raises(sgl.SGLError) as ei:
        p.set_points(gpu(inputs.points_gaussian(11, 2)))
    assert ei.value.status == 1


def test_host_buffers_match_device_path():
    B, M = 10, 800
    c, x, y = case(B, M, 7300)
    p = plan_for(B, M, host_io=True, x=x)
    f_dev = p.forward(gpu(c)).cpu().numpy()
    a_dev = p.adjoint(gpu(y)).cpu().numpy()
    f_host = np.zeros(M, dtype=np.complex128)
    a_host = np.zeros(p.Nc, dtype=np.complex128)
    p.forward_host(np.ascontiguousarray(x), c, f_host)
    p.adjoint_host(np.ascontiguousarray(x), y, a_host)
    assert np.array_equal(f_host, f_dev)
    assert rel(a_host, a_dev) <= 1e-13        # spreading order may differ between runs


def test_runs_on_a_side_stream():
    B, M = 8, 600
    c, x, y = case(B, M, 7400)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        p = plan_for(B, M, x=x)
        f = p.forward(gpu(c))
    s.synchronize()
    f_ref, _ = direct.forward(B, x, c)
    assert rel(f.cpu().numpy(), f_ref) <= 1e-10


@pytest.mark.parametrize("sigma", [1.5, 2.5, 3.0])
def test_other_oversampling_factors(sigma):
    B, M = 10, 500
    c, x, _ = case(B, M, 7500)
    p = plan_for(B, M, sigma=sigma, x=x)
    f = p.forward(gpu(c)).cpu().numpy()
    f_ref, _ = direct.forward(B, x, c)
    assert rel(f, f_ref) <= (1e-6 if sigma < 2 else 1e-10)


@pytest.mark.parametrize("prec,simt,ftol", [(sgl.PREC_FP64, False, 1e-12), (sgl.PREC_FP32_MIXED, False, 3e-6),
                                            (sgl.PREC_FP32_MIXED, True, 3e-6)])
def test_forward_grad_equals_separate_calls(prec, simt, ftol):
    # one pass gives the forward values and the point gradient of the separate calls
    B, M = 16, 2345
    c, x, _ = case(B, M, 9100)
    g = inputs.complex_normal(M, 9101)
    p = plan_for(B, M, prec=prec, x=x, simt=simt)
    f, gx = p.forward_grad(gpu(c), gpu(g))
    f, gx = f.cpu().numpy(), gx.cpu().numpy()
    assert rel(f, p.forward(gpu(c)).cpu().numpy()) <= ftol
    assert np.array_equal(gx, p.grad_points(gpu(c), gpu(g)).cpu().numpy())
    f_ref, _ = direct.forward(B, x, c)
    # FP32: measured 3.8e-7 (tensor cores) and 9.1e-7 (CUDA cores)
    check("forward_grad B=16 prec=%d simt=%d" % (prec, simt), rel(f, f_ref), 1e-10 if prec == sgl.PREC_FP64 else 5e-6)


def test_forward_grad_host_buffers():
    B, M = 10, 700
    c, x, _ = case(B, M, 9200)
    g = inputs.complex_normal(M, 9201)
    p = plan_for(B, M, host_io=True)
    vals = np.empty(M, dtype=np.complex128)
    gxyz = np.empty((M, 3))
    p.forward_grad_host(np.ascontiguousarray(x), c, g, vals, gxyz)
    p.set_points(gpu(x))
    f_dev, g_dev = p.forward_grad(gpu(c), gpu(g))
    assert np.allclose(vals, f_dev.cpu().numpy(), rtol=0, atol=1e-13 * np.abs(vals).max())
    assert np.allclose(gxyz, g_dev.cpu().numpy(), rtol=0, atol=1e-12 * np.abs(gxyz).max())


@pytest.mark.parametrize("q", [4, 8])
def test_double_float_and_binary64_loops_agree(q):
    # the FP64 plan's double-float hot loops and FFT passes (relative rounding ~2^-48 per
    # operation) against the binary64 ones of SGL_FLAG_NATIVE_FP64 (same window, so the same
    # approximation), on a size with many points per bin and tile; q = 4 and 8 take the two
    # spreading-kernel sizes.  Measured: adjoint 2.1e-13 (the FFT passes; 1.1e-13 with
    # binary64 FFT passes), the rest below 1e-13.
    B, M = 16, 20000
    c, x, y = case(B, M, 5100)
    g = y[::-1].copy()
    out = {}
    for native in (False, True):
        p = plan_for(B, M, q=q, x=x, native_fp64=native)
        f = p.forward(gpu(c)).cpu().numpy()
        a = p.adjoint(gpu(y)).cpu().numpy()
        fv, gx = p.forward_grad(gpu(c), gpu(g))
        out[native] = (f, a, fv.cpu().numpy(), gx.cpu().numpy())
        p.close()
    for k, tol in zip(range(4), (2e-13, 6e-13, 2e-13, 1e-11)):
        assert rel(out[False][k], out[True][k]) <= tol


@pytest.mark.parametrize("B", [10, 16])
@pytest.mark.parametrize("scale", [1e-200, 1e-30, 1e40, 1e200])
def test_fp64_plan_is_linear_over_the_whole_binary64_range(scale, B):
    # the double-float loops and FFT passes work on power-of-two scaled data, so magnitudes far
    # outside the binary32 range (the SGL polynomials reach 1e15 at r ~ 9 for B = 16) keep full
    # accuracy; B = 16 takes the double-float register FFT (lengths 128, 64), B = 10 the generic
    # kernel in binary64 (lengths 80, 40)
    M = 3000
    c, x, y = case(B, M, 5200)
    p = plan_for(B, M, x=x)
    f1 = p.forward(gpu(c)).cpu().numpy()
    a1 = p.adjoint(gpu(y)).cpu().numpy()
    fs = p.forward(gpu(c * scale)).cpu().numpy()
    as_ = p.adjoint(gpu(y * scale)).cpu().numpy()
    _, gs = p.forward_grad(gpu(c * scale), gpu(y))
    _, g1 = p.forward_grad(gpu(c), gpu(y))
    assert np.isfinite(fs).all() and np.isfinite(as_).all()
    assert rel(fs / scale, f1) <= 3e-13
    assert rel(as_ / scale, a1) <= 3e-13
    assert rel(gs.cpu().numpy() / scale, g1.cpu().numpy()) <= 1e-11


def test_host_calls_reuse_the_points_when_xyz_is_none():
    B, M = 8, 1500
    c, x, y = case(B, M, 5300)
    g = y[::-1].copy()
    p = plan_for(B, M, host_io=True)
    vals, gxyz = np.zeros(M, complex), np.zeros((M, 3))
    p.forward_grad_host(np.ascontiguousarray(x), c, g, vals, gxyz)
    a_host = np.zeros(p.Nc, complex)
    p.adjoint_host(None, y, a_host)                 # the points of the previous call
    f2 = np.zeros(M, complex)
    p.forward_host(None, c, f2)
    q = plan_for(B, M, x=x)
    assert rel(a_host, q.adjoint(gpu(y)).cpu().numpy()) <= 1e-12
    assert rel(f2, q.forward(gpu(c)).cpu().numpy()) <= 1e-12
    # reusing the points with another M is an argument error (SGL_ERR_ARG = 1)
    assert p.lib.sgl_adjoint_host(p._h, None, M - 1, y.ctypes.data, a_host.ctypes.data) == 1
    fresh = plan_for(B, M, host_io=True)
    with pytest.raises(sgl.SGLError):
        fresh.adjoint_host(None, y, a_host)            # no points set yet
