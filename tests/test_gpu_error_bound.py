"""Error control on the GPU (marked gpu): measured FP64 errors against the oracle's direct sums
stay below plan.error_bound() * plan.eta_l1(coef); the observations of Sect. 7 / the tests of
Sect. 8 on the error vs the spreading radius kappa and vs the bandwidth B (points uniform in the
ball of radius kappa, as there), at a cutoff where the NFFT error is far above rounding."""
import numpy as np
import pytest
import torch

import paper_1809_10786_gb300 as sgl
from paper_1809_10786_gb300 import inputs
from oracle import direct

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def measured_and_bound(B, x, c, q, window=sgl.WIN_KB):
    p = sgl.Plan(B, len(x), precision=sgl.PREC_FP64, window=window, q=q, device=DEV)
    p.set_points(gpu(x))
    f = p.forward(gpu(c)).cpu().numpy()
    bound = p.error_bound() * p.eta_l1(gpu(c))
    p.close()
    ref, _ = direct.forward(B, x, c)
    return float(np.abs(f - ref).max()), bound, float(np.abs(ref).max())


@pytest.mark.parametrize("B,q,window", [(8, 3, sgl.WIN_KB), (16, 4, sgl.WIN_KB), (12, 5, sgl.WIN_GAUSS),
                                        (20, 6, sgl.WIN_KB), (10, 8, sgl.WIN_KB)])
def test_forward_error_below_the_bound(B, q, window):
    x = inputs.points_gaussian(2000, 7000 + B)
    c = inputs.coefficients(B, 7100 + B)
    err, bound, fmax = measured_and_bound(B, x, c, q, window)
    assert err <= bound + 1e-12 * fmax          # slack: binary64 rounding of the fast path itself


def test_plan_bound_equals_the_parameter_bound():
    p = sgl.Plan(12, 10, precision=sgl.PREC_FP64, q=5, sigma=2.5, device=DEV)
    assert p.error_bound() == sgl.nfft_error_bound(12, sgl.WIN_KB, 5, 2.5)
    p.close()


@pytest.mark.parametrize("q", [4, 6])
def test_error_grows_with_the_spreading_radius(q):
    # Sect. 8 (error vs kappa), B = 32, M = 1000 uniform in the ball of radius kappa: the bound
    # holds at every kappa and the error grows with kappa (Sect. 7: rho enters as e^{rho^2 / 2}).
    # Prints one row per kappa (run with -s for the table).
    B = 32
    c = inputs.coefficients(B, 7200)
    errs = []
    for kappa in (1.0, 2.0, 3.0, 4.0, 5.0):
        x = inputs.points_ball(1000, 7201, radius=kappa)
        err, bound, fmax = measured_and_bound(B, x, c, q)
        print("\nerror vs kappa: q=%d B=%d kappa=%.0f  max abs error %.2e  bound*||eta||_1 %.2e  max|f| %.2e"
              % (q, B, kappa, err, bound, fmax), end="")
        assert err <= bound + 1e-12 * fmax
        errs.append(err)
    assert errs[-1] > 10 * errs[0]


@pytest.mark.parametrize("q", [4, 6])
def test_error_grows_slowly_with_the_bandwidth(q):
    # Sect. 8 (error vs B), kappa = 5: the bound holds and the error grows with B (-s prints the rows)
    x = inputs.points_ball(1000, 7301, radius=5.0)
    errs = []
    for B in (8, 16, 24, 32, 48):
        err, bound, fmax = measured_and_bound(B, x, inputs.coefficients(B, 7300 + B), q)
        print("\nerror vs B: q=%d kappa=5 B=%d  max abs error %.2e  bound*||eta||_1 %.2e  max|f| %.2e"
              % (q, B, err, bound, fmax), end="")
        assert err <= bound + 1e-12 * fmax
        errs.append(err)
    assert errs[-1] > errs[0]


def test_chosen_cutoff_meets_a_target_accuracy():
    # pick q for a target error per unit ||eta||_1, then check the transform against the oracle
    B, tol = 16, 1e-9
    q = sgl.choose_cutoff(B, tol)
    x = inputs.points_gaussian(1500, 7400)
    c = inputs.coefficients(B, 7401)
    p = sgl.Plan(B, len(x), precision=sgl.PREC_FP64, q=q, device=DEV)
    p.set_points(gpu(x))
    l1 = p.eta_l1(gpu(c))
    f = p.forward(gpu(c)).cpu().numpy()
    p.close()
    ref, _ = direct.forward(B, x, c)
    assert np.abs(f - ref).max() <= tol * l1 + 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("M,tol", [(1500, 1e-9), (1500, 1e-5)])
def test_chosen_sigma_and_cutoff_meet_a_target_accuracy(M, tol):
    # (sigma, q) from the cost model and the bound; the plan built with them meets tol per unit ||eta||_1
    B = 16
    sigma, q, _ = sgl.choose_params(B, M, tol, precision=sgl.PREC_FP64)
    x = inputs.points_gaussian(M, 7500)
    c = inputs.coefficients(B, 7501)
    p = sgl.Plan(B, M, precision=sgl.PREC_FP64, q=q, sigma=sigma, device=DEV)
    assert p.error_bound() <= tol
    p.set_points(gpu(x))
    l1 = p.eta_l1(gpu(c))
    f = p.forward(gpu(c)).cpu().numpy()
    p.close()
    ref, _ = direct.forward(B, x, c)
    assert np.abs(f - ref).max() <= tol * l1 + 1e-12 * np.abs(ref).max()
