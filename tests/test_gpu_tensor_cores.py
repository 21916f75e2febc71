"""Tensor-core (tcgen05) interpolation and gradient of FP32-mixed plans (marked gpu).

FP32-mixed plans with q <= 8 and windowed axes 0 and 1 run the windowed interpolation and
the window-derivative gradient as slab products on the tensor cores (3xTF32 split, FP32
accumulation).  Checked here against the oracle's direct sums (same envelopes as the
CUDA-core kernels) and against the CUDA-core kernels of the same plan type (SGL_FLAG_SIMT),
on inputs that span many super-bins, super-bins with several 128-point chunks, a ragged
last chunk, both windows and several cutoffs.
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


def clustered(M, seed, centre=(0.3, -0.2, 0.1), width=0.05):
    """Points packed into a few grid cells: super-bins with several 128-point chunks."""
    rng = np.random.default_rng(seed)
    return np.asarray(centre) + width * rng.standard_normal((M, 3))


def well_conditioned(x, rho):
    """Points away from the origin and the polar axis (t0 and theta away from 0 and pi)."""
    r = np.linalg.norm(x, axis=1)
    sin_theta = np.hypot(x[:, 0], x[:, 1]) / np.maximum(r, 1e-300)
    return (r > 0.05 * rho) & (r < 0.95 * rho) & (sin_theta > 0.1)


def pair(B, M, q, win, x):
    tc = sgl.Plan(B, M, precision=sgl.PREC_FP32_MIXED, window=win, q=q, device=DEV, tensor_cores=True)
    ref = sgl.Plan(B, M, precision=sgl.PREC_FP32_MIXED, window=win, q=q, device=DEV, simt=True)
    for p in (tc, ref):
        p.set_points(gpu(x))
    return tc, ref


# bounds against the oracle, about 5x the errors measured on GB300 (forward / gradient on the
# well-conditioned points): q = 8 KB 3.4e-7 / 3.9e-7, q = 6 3.7e-7 / 2.2e-7, q = 4 2.1e-7 / 3.1e-6,
# q = 8 Gauss 2.5e-7 / 5.6e-7; at q = 2 the window approximation error itself dominates (forward
# 9.5e-4, gradient 1.3e-2, amplified by the chain rule)
@pytest.mark.parametrize("B,M,q,win,bound,gbound", [
    (16, 3001, 8, sgl.WIN_KB, 2e-6, 2e-6),
    (20, 2500, 6, sgl.WIN_KB, 2e-6, 1.2e-6),
    (24, 4099, 4, sgl.WIN_KB, 1.2e-6, 1.5e-5),
    (16, 1777, 2, sgl.WIN_KB, 2e-3, 5e-2),
    (16, 2000, 8, sgl.WIN_GAUSS, 1.5e-6, 3e-6),
])
def test_tc_forward_and_gradient_match_oracle(B, M, q, win, bound, gbound):
    c = inputs.coefficients(B, 8100 + B)
    x = inputs.points_gaussian(M, 8101 + B)
    g = inputs.complex_normal(M, 8102 + B)
    tc, ref = pair(B, M, q, win, x)
    assert tc.info()["tensor_cores"] == {"interp": True, "grad": True, "spread": False}
    assert ref.info()["tensor_cores"] == {"interp": False, "grad": False, "spread": False}
    f = tc.forward(gpu(c)).cpu().numpy()
    gx = tc.grad_points(gpu(c), gpu(g)).cpu().numpy()
    tc.sync()
    f_simt = ref.forward(gpu(c)).cpu().numpy()
    gx_simt = ref.grad_points(gpu(c), gpu(g)).cpu().numpy()
    f_ref, _ = direct.forward(B, x, c)
    g_ref, _ = direct.grad_points(B, x, c, g)
    # forward: the two FP32 kernels agree to FP32 rounding, and both sit in the envelope
    check("tc vs simt forward B=%d q=%d win=%d" % (B, q, win), rel(f, f_simt), 6e-6)     # measured <= 1.3e-6
    check("tc forward B=%d q=%d win=%d" % (B, q, win), rel(f, f_ref), bound)
    # gradient: the chain rule's 1/(r sin theta) amplifies FP32 rounding near the axis and the
    # origin differently for the two summation orders, so each is held to the oracle instead
    # (and at q = 2 the window's approximation error itself is amplified by dt0/dr = -2 / (rho
    # sin t0) near the origin, so the oracle comparison takes the well-conditioned points)
    ok = well_conditioned(x, tc.rho())
    e_tc, e_simt = rel(gx[ok], g_ref[ok]), rel(gx_simt[ok], g_ref[ok])
    check("tc gradient B=%d q=%d win=%d" % (B, q, win), e_tc, gbound)
    assert e_tc <= 3 * e_simt + 1e-6, (e_tc, e_simt)
    # over all points, near-axis ones included (measured up to 1.2e-3: 1/(r sin theta) amplification)
    check("tc vs simt gradient B=%d q=%d win=%d" % (B, q, win), rel(gx, gx_simt), 5e-3)


# adjoint against the oracle: measured 4.0e-7, 1.9e-7, 2.7e-7, 2.6e-7
@pytest.mark.parametrize("B,M,q,win,bound", [
    (16, 3001, 8, sgl.WIN_KB, 2e-6),
    (20, 2500, 6, sgl.WIN_KB, 1e-6),
    (24, 4099, 4, sgl.WIN_KB, 1.5e-6),
    (16, 2000, 8, sgl.WIN_GAUSS, 1.5e-6),
])
def test_tc_adjoint_matches_oracle(B, M, q, win, bound):
    y = inputs.values(M, 8150 + B)
    x = inputs.points_gaussian(M, 8151 + B)
    tc, ref = pair(B, M, q, win, x)
    a = tc.adjoint(gpu(y)).cpu().numpy()
    tc.sync()
    a_simt = ref.adjoint(gpu(y)).cpu().numpy()
    a_ref, _ = direct.adjoint(B, x, y)
    check("tc vs simt adjoint B=%d q=%d win=%d" % (B, q, win), rel(a, a_simt), 2e-6)      # measured <= 3.6e-7
    check("tc adjoint B=%d q=%d win=%d" % (B, q, win), rel(a, a_ref), bound)
    check("simt adjoint B=%d q=%d win=%d" % (B, q, win), rel(a_simt, a_ref), bound)
    # the adjoint pair stays an adjoint pair to FP32 rounding
    c = inputs.coefficients(B, 8152 + B)
    f = tc.forward(gpu(c)).cpu().numpy()
    check("tc adjoint identity B=%d q=%d" % (B, q), abs(np.vdot(y, f) - np.vdot(a, c)) / (np.linalg.norm(f) * np.linalg.norm(y)), 2e-8)


def test_tc_dense_super_bins_and_ragged_chunks():
    # ~6000 points in a few cells: several 128-point chunks per super-bin, ragged last chunks
    B, M = 16, 6007
    c = inputs.coefficients(B, 8200)
    x = clustered(M, 8201)
    g = inputs.complex_normal(M, 8202)
    tc, ref = pair(B, M, 8, sgl.WIN_KB, x)
    f = tc.forward(gpu(c)).cpu().numpy()
    gx = tc.grad_points(gpu(c), gpu(g)).cpu().numpy()
    tc.sync()
    assert rel(f, ref.forward(gpu(c)).cpu().numpy()) <= 2e-6
    gx_simt = ref.grad_points(gpu(c), gpu(g)).cpu().numpy()
    idx = inputs.subset(M, 300, 8203)
    f_ref, _ = direct.forward(B, x[idx], c)
    g_ref, _ = direct.grad_points(B, x[idx], c, g[idx])
    check("tc dense forward", rel(f[idx], f_ref), 2e-6)                  # measured 4.3e-7
    check("tc dense gradient", rel(gx[idx], g_ref), 3e-6)                # measured 6.5e-7
    assert rel(gx[idx], g_ref) <= 3 * rel(gx_simt[idx], g_ref) + 1e-6
    # spreading with several 32-point chunks per super-bin
    y = inputs.values(M, 8204)
    # spreading of crowded super-bins (several entries of the work list each) against the oracle
    a_ref, _ = direct.adjoint(B, x, y)
    check("dense adjoint", rel(tc.adjoint(gpu(y)).cpu().numpy(), a_ref), 6e-7)           # measured 1.2e-7


@pytest.mark.parametrize("M", [1, 127, 128, 129])
def test_tc_small_point_counts(M):
    B = 12
    c = inputs.coefficients(B, 8300 + M)
    x = inputs.points_gaussian(M, 8301 + M)
    tc, ref = pair(B, M, 8, sgl.WIN_KB, x)
    f = tc.forward(gpu(c)).cpu().numpy()
    tc.sync()
    f_ref, _ = direct.forward(B, x, c)
    assert rel(f, ref.forward(gpu(c)).cpu().numpy()) <= 2e-6
    check("tc small M=%d forward" % M, rel(f, f_ref), 2.5e-6)              # measured <= 4.5e-7


def test_tc_is_used_only_where_eligible():
    # FP64 plans, q > 8 and grids whose axis 1 is not windowed stay on the CUDA-core kernels
    none = {"interp": False, "grad": False, "spread": False}
    f32 = sgl.PREC_FP32_MIXED
    assert sgl.Plan(16, 10, precision=sgl.PREC_FP64, device=DEV, tensor_cores=True).info()["tensor_cores"] == none
    assert sgl.Plan(16, 10, precision=f32, q=9, device=DEV, tensor_cores=True).info()["tensor_cores"] == none
    assert sgl.Plan(8, 10, precision=f32, q=8, device=DEV, tensor_cores=True).info()["tensor_cores"] == none
    # default choice: the faster kernels (tensor cores from q = 6 on)
    both = {"interp": True, "grad": True, "spread": False}
    assert sgl.Plan(16, 10, precision=f32, q=8, device=DEV).info()["tensor_cores"] == both
    assert sgl.Plan(16, 10, precision=f32, q=6, device=DEV).info()["tensor_cores"] == both
    assert sgl.Plan(16, 10, precision=f32, q=4, device=DEV).info()["tensor_cores"] == none
