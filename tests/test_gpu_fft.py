"""The register FFT kernels (power-of-two lengths 64 ... 1024) against the generic mixed-radix
kernel, the double-float passes of FP64 plans against binary64 ones, and both against the oracle
(marked gpu).

Both kernels compute the same pruned transforms of the NFFT (Sect. 2) in different orders, so
their forward values and adjoint coefficients agree to rounding.  At sigma = 2 the grid lengths
are (8B, 4B, 4B): B = 8 runs lengths 64 (register) and 32 (generic), B = 16 lengths 128 and 64,
B = 32 lengths 256 and 128, B = 64 lengths 512 and 256; B = 12 (96, 48) stays generic on every
axis.  The bounds are a few times the measured differences (checked through `envelope`).
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


def run(B, M, prec, generic, seed, native=False):
    c = inputs.coefficients(B, seed)
    x = inputs.points_gaussian(M, seed + 1)
    y = inputs.values(M, seed + 2)
    p = sgl.Plan(B, M, precision=prec, q=8, device=DEV, generic_fft=generic, native_fp64=native)
    p.set_points(gpu(x))
    f = p.forward(gpu(c)).cpu().numpy()
    a = p.adjoint(gpu(y)).cpu().numpy()
    return f, a, (c, x, y)


# FP64 plans: double-float passes (default) or binary64 ones (native_fp64) in both kernels;
# FP32-mixed: binary32 angular passes and a double-float radial pass in both
@pytest.mark.parametrize("B", [8, 16, 32, 64])
@pytest.mark.parametrize("prec,native,tol", [(sgl.PREC_FP64, False, 2e-12), (sgl.PREC_FP64, True, 1e-13),
                                             (sgl.PREC_FP32_MIXED, False, 2e-6)])
def test_register_fft_matches_generic(B, prec, native, tol):
    M = 3000
    f_r, a_r, _ = run(B, M, prec, False, 9400 + B, native)
    f_g, a_g, _ = run(B, M, prec, True, 9400 + B, native)
    check("fft reg vs generic forward B=%d prec=%d native=%d" % (B, prec, native), rel(f_r, f_g), tol)
    check("fft reg vs generic adjoint B=%d prec=%d native=%d" % (B, prec, native), rel(a_r, a_g), tol)


@pytest.mark.parametrize("B", [16, 64])
def test_double_float_fft_matches_binary64(B):
    # FP64 plans: the double-float passes (and windowed loops) against the binary64 ones
    f_d, a_d, _ = run(B, 3000, sgl.PREC_FP64, False, 9600 + B, False)
    f_n, a_n, _ = run(B, 3000, sgl.PREC_FP64, False, 9600 + B, True)
    check("fft double-float vs binary64 forward B=%d" % B, rel(f_d, f_n), 2e-12)
    check("fft double-float vs binary64 adjoint B=%d" % B, rel(a_d, a_n), 2e-12)


@pytest.mark.parametrize("B,prec,tol", [(16, sgl.PREC_FP64, 1e-10), (32, sgl.PREC_FP64, 1e-10),
                                        (32, sgl.PREC_FP32_MIXED, 3e-6), (12, sgl.PREC_FP64, 1e-10)])
def test_register_fft_against_the_oracle(B, prec, tol):
    M = 400
    f, a, (c, x, y) = run(B, M, prec, False, 9500 + B)
    ref, _ = direct.forward(B, x, c)
    check("fft oracle forward B=%d prec=%d" % (B, prec), rel(f, ref), tol)
    aref, _ = direct.adjoint(B, x, y)
    check("fft oracle adjoint B=%d prec=%d" % (B, prec), rel(a, aref), tol)

