"""Differentiation through torch.autograd (marked gpu): the differentiation workload
(B = 32, M = 2e5 points, targets y = f_true(x) + 0.01 complex noise, loss
sum |f(x_j) - y_j|^2).  Gradients with respect to the coefficients (through the
adjoint) and to the point coordinates (window-derivative interpolation) are checked
against the oracle's direct gradient on a 1000-point subset (the loss restricted to
it) and against central finite differences of the GPU loss (h = 1e-6)."""
import numpy as np
import pytest
import torch

import paper_1809_10786_gb300 as sgl
from envelope import check
from paper_1809_10786_gb300 import inputs
from paper_1809_10786_gb300.autograd import ndsglft
from oracle import direct

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


@pytest.fixture(scope="module")
def workload():
    B, M = 32, 200_000
    c_true = inputs.coefficients(B, inputs.seed_for(4))
    c0 = inputs.coefficients(B, inputs.seed_for(4) + 1)          # starting coefficients: an independent draw
    x = inputs.points_gaussian(M, inputs.seed_for(4, 1))
    noise = inputs.complex_normal(M, inputs.seed_for(4, 2), scale=0.01)
    idx = inputs.subset(M, 1000, inputs.seed_for(4, 3))
    mask = np.zeros(M)
    mask[idx] = 1.0
    f_true, _ = direct.forward(B, x[idx], c_true)
    y = np.zeros(M, dtype=np.complex128)
    y[idx] = f_true + noise[idx]
    return B, M, c0, x, y, idx, mask


def masked_loss(plan, c, x, y, mask):
    f = ndsglft(c, x, plan)
    r = (f - y) * mask
    return (r.real ** 2 + r.imag ** 2).sum()


# FP32-mixed: about 5x the measured 2.0e-7 (coefficients) and 9.5e-7 (points)
@pytest.mark.parametrize("prec,tol_c,tol_x", [(sgl.PREC_FP64, 1e-9, 1e-8), (sgl.PREC_FP32_MIXED, 1e-6, 5e-6)])
def test_gradients_against_oracle(workload, prec, tol_c, tol_x):
    B, M, c0, x, y, idx, mask = workload
    plan = sgl.Plan(B, M, precision=prec, q=8)
    c = torch.from_numpy(c0).to(DEV).requires_grad_(True)
    xt = torch.from_numpy(x).to(DEV).requires_grad_(True)
    loss = masked_loss(plan, c, xt, torch.from_numpy(y).to(DEV), torch.from_numpy(mask).to(DEV))
    loss.backward()
    gc = c.grad.cpu().numpy()
    gx = xt.grad.cpu().numpy()
    # oracle: residual on the subset, grad_c = 2 Lambda^H r, grad_x = 2 Re(conj(r) df/dx)
    f_sub, _ = direct.forward(B, x[idx], c0)
    r = f_sub - y[idx]
    gc_ref, _ = direct.adjoint(B, x[idx], 2 * r)
    gx_ref, _ = direct.grad_points(B, x[idx], c0, 2 * r)
    check("autograd coefficients prec=%d" % prec, np.abs(gc - gc_ref).max() / np.abs(gc_ref).max(), tol_c)
    check("autograd points prec=%d" % prec, np.abs(gx[idx] - gx_ref).max() / np.abs(gx_ref).max(), tol_x)
    others = np.setdiff1d(np.arange(M), idx)
    assert np.abs(gx[others]).max() == 0.0


def test_gradients_against_finite_differences(workload):
    B, M, c0, x, y, idx, mask = workload
    plan = sgl.Plan(B, M, precision=sgl.PREC_FP64, q=8)
    yt, mt = torch.from_numpy(y).to(DEV), torch.from_numpy(mask).to(DEV)
    c = torch.from_numpy(c0).to(DEV).requires_grad_(True)
    xt = torch.from_numpy(x).to(DEV).requires_grad_(True)
    masked_loss(plan, c, xt, yt, mt).backward()
    gc = c.grad.cpu().numpy()
    gx = xt.grad.cpu().numpy()
    h = 1e-6
    rng = np.random.default_rng(7)

    def L(cc, xx):
        with torch.no_grad():
            return float(masked_loss(plan, torch.from_numpy(cc).to(DEV), torch.from_numpy(xx).to(DEV), yt, mt))

    # 32 coefficient components, real and imaginary parts
    for k in rng.choice(len(c0), 16, replace=False):
        for unit in (1.0, 1j):
            cp, cm = c0.copy(), c0.copy()
            cp[k] += h * unit
            cm[k] -= h * unit
            fd = (L(cp, x) - L(cm, x)) / (2 * h)
            an = gc[k].real if unit == 1.0 else gc[k].imag
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)) + 1e-5 * np.abs(gc).max(), (k, unit, fd, an)
    # point coordinates of subset points away from the outermost radius (rho stays fixed)
    r = np.linalg.norm(x, axis=1)
    cand = [i for i in idx if r[i] < 0.9 * r.max()][:8]
    for i in cand:
        for d in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, d] += h
            xm[i, d] -= h
            fd = (L(c0, xp) - L(c0, xm)) / (2 * h)
            assert abs(fd - gx[i, d]) <= 1e-5 * max(1.0, abs(gx[i, d])) + 1e-6 * np.abs(gx).max(), (i, d, fd, gx[i, d])
