"""FP32 spreading, the first step of the adjoint NFFT (Sect. 2), against the oracle (marked gpu).

Wherever axis 1 of the grid is windowed the FP32 plans spread with the sliding-window kernel:
each work-list entry's points are sorted by their first azimuthal tap and swept through a window
of 16 (2q <= 8: 8) tile columns per slab, retiring columns as it moves.  These cases stress what
that sort and window depend on: a crowded super-bin split over several entries (thousands of
points, most sharing their first tap), every first tap of a chunk, both windows and every
cutoff.  The bounds are a few times the measured errors (`envelope`).
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


def adjoint(B, x, y, q, win=sgl.WIN_KB):
    p = sgl.Plan(B, len(x), precision=sgl.PREC_FP32_MIXED, window=win, q=q, device=DEV)
    p.set_points(gpu(x))
    a = p.adjoint(gpu(y)).cpu().numpy()
    p.close()
    return a


def test_crowded_super_bin_over_several_entries():
    # 3000 points within 1e-3 of one point: one super-bin, three work-list entries of <= 1024
    rng = np.random.default_rng(9300)
    x = np.array([1.0, 0.5, 0.3]) + 1e-3 * rng.standard_normal((3000, 3))
    x = np.concatenate([x, inputs.points_gaussian(200, 9301)], 0)   # rho and a few other bins
    y = inputs.values(len(x), 9302)
    a = adjoint(16, x, y, 8)
    ref, _ = direct.adjoint(16, x, y)
    check("spread crowded super-bin B=16 q=8", rel(a, ref), 5e-7)


@pytest.mark.parametrize("q", [4, 6, 8])
def test_every_first_tap_of_a_chunk(q):
    # points at azimuth phi = 2 pi (k + 0.5) / N2 for every cell k: every first tap s of every chunk
    B = 16
    n2 = 4 * B * 2                                   # N2 at sigma = 2
    k = np.arange(n2)
    phi = 2 * np.pi * (k + 0.5) / n2
    r, th = 1.2, 1.1
    x = np.stack([r * np.sin(th) * np.cos(phi), r * np.sin(th) * np.sin(phi), np.full(n2, r * np.cos(th))], 1)
    x = np.concatenate([x, inputs.points_gaussian(500, 9400 + q)], 0)
    y = inputs.values(len(x), 9410 + q)
    a = adjoint(B, x, y, q)
    ref, _ = direct.adjoint(B, x, y)
    check("spread every first tap B=16 q=%d" % q, rel(a, ref), 5e-7)


@pytest.mark.parametrize("q", [4, 8])
def test_gaussian_window(q):
    # against the FP64 plan with the same window and cutoff (the Gaussian window's own error at
    # q = 4 is far above the FP32 rounding, so the oracle would not see a spreading slip there)
    B, M = 24, 2000
    x = inputs.points_gaussian(M, 9500 + q)
    y = inputs.values(M, 9510 + q)
    a = adjoint(B, x, y, q, sgl.WIN_GAUSS)
    p = sgl.Plan(B, M, precision=sgl.PREC_FP64, window=sgl.WIN_GAUSS, q=q, device=DEV)
    p.set_points(gpu(x))
    ref = p.adjoint(gpu(y)).cpu().numpy()
    check("spread gaussian vs FP64 plan B=24 q=%d" % q, rel(a, ref), 5e-7)
