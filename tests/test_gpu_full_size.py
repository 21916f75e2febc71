"""Parity at the workload sizes (marked gpu), in the launch configuration bench.py times.

The oracle evaluates sampled outputs one by one: forward values and gradients at
sampled points, and the adjoint of values that are zero outside the sample (the
adjoint is linear, so this checks the full-size spreading and FFT path against a
sum the oracle can form).  The adjoint identity is checked on all points.
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


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.fixture(scope="module")
def workload_b32():
    B, M = 32, 100_000
    c = inputs.coefficients(B, inputs.seed_for(1), scale_by_degree=True)
    x = inputs.points_gaussian(M, inputs.seed_for(1, 1))
    y = inputs.values(M, inputs.seed_for(1, 2))
    idx = inputs.subset(M, 2000, inputs.seed_for(1, 3))
    return B, M, c, x, y, idx


@pytest.fixture(scope="module")
def workload_b64():
    B, M = 64, 1_000_000
    c = inputs.coefficients(B, inputs.seed_for(2))
    x = inputs.points_gaussian(M, inputs.seed_for(2, 1))
    y = inputs.values(M, inputs.seed_for(2, 100))
    g = inputs.complex_normal(M, inputs.seed_for(2, 200))
    idx = inputs.subset(M, 5000, inputs.seed_for(2, 3))        # the workload's oracle subset
    return B, M, c, x, y, g, idx


# FP32-mixed bounds: about 5x the errors measured on GB300 (forward 4.1e-7, adjoint 5.3e-8,
# adjoint identity 1.1e-9 relative to |f| |y|)
@pytest.mark.parametrize("prec,tol_f,tol_a", [(sgl.PREC_FP64, 1e-10, 1e-10), (sgl.PREC_FP32_MIXED, 2e-6, 3e-7)])
def test_b32_m1e5_forward_adjoint(workload_b32, prec, tol_f, tol_a):
    B, M, c, x, y, idx = workload_b32
    p = sgl.Plan(B, M, precision=prec, q=8)
    p.set_points(gpu(x))
    f = p.forward(gpu(c)).cpu().numpy()
    f_ref, _ = direct.forward(B, x[idx], c)
    check("b32 m1e5 forward prec=%d" % prec, rel(f[idx], f_ref), tol_f)
    a_all = p.adjoint(gpu(y)).cpu().numpy()
    lhs, rhs = np.vdot(y, f), np.vdot(a_all, c)
    check("b32 m1e5 adjoint identity prec=%d" % prec, abs(lhs - rhs) / (np.linalg.norm(f) * np.linalg.norm(y)),
          1e-12 if prec == sgl.PREC_FP64 else 5e-9)
    ym = np.zeros_like(y)
    ym[idx] = y[idx]
    a = p.adjoint(gpu(ym)).cpu().numpy()
    a_ref, _ = direct.adjoint(B, x[idx], y[idx])
    check("b32 m1e5 adjoint prec=%d" % prec, rel(a, a_ref), tol_a)


# FP32-mixed bounds about 5x the errors measured on GB300 (5000-point subset; forward / adjoint /
# gradient): q = 8: 4.2e-7 / 7.0e-8 / 8.2e-7; q = 6: 2.3e-7 / 6.4e-8 / 1.3e-6; q = 4: 4.8e-7 /
# 9.4e-8 / 3.1e-6
@pytest.mark.parametrize("prec,q,tol_f,tol_a,tol_g", [(sgl.PREC_FP64, 8, 1e-10, 1e-10, 1e-8),
                                                      (sgl.PREC_FP32_MIXED, 8, 2e-6, 3.5e-7, 4e-6),
                                                      (sgl.PREC_FP32_MIXED, 6, 1.2e-6, 3e-7, 7e-6),
                                                      (sgl.PREC_FP32_MIXED, 4, 2.5e-6, 5e-7, 1.5e-5)])
def test_b64_m1e6_sampled(workload_b64, prec, q, tol_f, tol_a, tol_g):
    B, M, c, x, y, g, idx = workload_b64
    p = sgl.Plan(B, M, precision=prec, q=q)
    p.set_points(gpu(x))
    f = p.forward(gpu(c)).cpu().numpy()
    f_ref, _ = direct.forward(B, x[idx], c)
    ef = rel(f[idx], f_ref)
    ym = np.zeros_like(y)
    ym[idx] = y[idx]
    a = p.adjoint(gpu(ym)).cpu().numpy()
    a_ref, _ = direct.adjoint(B, x[idx], y[idx])
    ea = rel(a, a_ref)
    gx = p.grad_points(gpu(c), gpu(g)).cpu().numpy()
    g_ref, _ = direct.grad_points(B, x[idx], c, g[idx])
    eg = rel(gx[idx], g_ref)
    check("b64 m1e6 forward prec=%d q=%d" % (prec, q), ef, tol_f)
    check("b64 m1e6 adjoint prec=%d q=%d" % (prec, q), ea, tol_a)
    check("b64 m1e6 gradient prec=%d q=%d" % (prec, q), eg, tol_g)


def test_b64_m1e6_adjoint_identity_fp64(workload_b64):
    B, M, c, x, y, g, idx = workload_b64
    p = sgl.Plan(B, M, precision=sgl.PREC_FP64, q=8)
    p.set_points(gpu(x))
    f = p.forward(gpu(c)).cpu().numpy()
    a = p.adjoint(gpu(y)).cpu().numpy()
    assert abs(np.vdot(y, f) - np.vdot(a, c)) <= 1e-12 * np.linalg.norm(f) * np.linalg.norm(y)


# FP32-mixed: measured 5.5e-7
@pytest.mark.parametrize("prec,tol", [(sgl.PREC_FP64, 1e-9), (sgl.PREC_FP32_MIXED, 3e-6)])
def test_b32_m2e5_gradients(prec, tol):
    # differentiation workload: B = 32, M = 2e5, gradient checked on 1000 points
    B, M = 32, 200_000
    c = inputs.coefficients(B, inputs.seed_for(4))
    x = inputs.points_gaussian(M, inputs.seed_for(4, 1))
    g = inputs.complex_normal(M, inputs.seed_for(4, 2))
    idx = inputs.subset(M, 1000, inputs.seed_for(4, 3))
    p = sgl.Plan(B, M, precision=prec, q=8)
    p.set_points(gpu(x))
    gx = p.grad_points(gpu(c), gpu(g)).cpu().numpy()
    ref, _ = direct.grad_points(B, x[idx], c, g[idx])
    check("b32 m2e5 gradient prec=%d" % prec, rel(gx[idx], ref), tol)
