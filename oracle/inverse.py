"""Oracle of the inverse transform (iNFSGLFT): SGL Fourier coefficients from scattered samples.

TEST INFRASTRUCTURE ONLY: imported by tests/, never by the product path.

The paper builds the inverse transform as a conjugate-gradient method on the normal equations
with the fast transform and its adjoint (Sect. 2, end: the iNFFT; Sect. 7, end: the same for
the NFSGLFT).  Two cases:

  * M >= Nc, least squares min ||f - Lambda c||_2: normal equations of the first kind
    Lambda^H Lambda c = Lambda^H f, by CGNR (Golub and Van Loan, Alg. 10.4.1);
  * M < Nc, minimum-norm solution: Lambda Lambda^H g = f, c = Lambda^H g, by CGNE
    (Alg. 10.4.2).

Here Lambda is the dense matrix [H_mu(x_i)] built with the oracle's direct basis, and the
iterations follow the algorithms' steps in order, in float64 (the scalar coefficients alpha,
beta in numpy's longdouble, as the paper's test computed them in extended precision).

The initial guess of the paper's last test (Sect. 8) is the mid-point rule on the Cartesian
grid G_N = kappa [2j/N - 1, 2k/N - 1, 2l/N - 1]:  c_mu ~ h^3 sum_i f(x_i) conj(H_mu(x_i))
e^{-|x_i|^2}, h = 2 kappa / N the grid spacing (the printed factor 8 N^{-1} reads h^3 =
8 kappa^3 / N^3: the cell volume of the rule).
"""
import numpy as np

from . import direct


def matrix(B, xyz):
    """Lambda = [H_mu(x_i)] as complex128 [M, Nc] (Def. of the NDSGLFT)."""
    xyz = np.asarray(xyz, dtype=np.float64).reshape(-1, 3)
    return np.stack([direct.basis(B, x) for x in xyz]) if len(xyz) else np.zeros((0, direct.num_coeffs(B)), complex)


def _norm2(v):
    return np.longdouble(np.vdot(v, v).real)


def cgnr(L, f, c0, iters):
    """Alg. 10.4.1 on Lambda^H Lambda c = Lambda^H f; returns (c, residual norms ||f - Lambda c||)."""
    c = np.array(c0, dtype=np.complex128)
    r = f - L @ c
    z = L.conj().T @ r
    p = z.copy()
    zz = _norm2(z)
    res = [float(np.sqrt(_norm2(r)))]
    for _ in range(iters):
        if zz == 0:
            break
        w = L @ p
        alpha = zz / _norm2(w)
        c = c + complex(alpha) * p
        r = r - complex(alpha) * w
        z = L.conj().T @ r
        zz_new = _norm2(z)
        beta = zz_new / zz
        p = z + complex(beta) * p
        zz = zz_new
        res.append(float(np.sqrt(_norm2(r))))
    return c, res


def cgne(L, f, c0, iters):
    """Alg. 10.4.2 on Lambda Lambda^H g = f, c = Lambda^H g; returns (c, residual norms)."""
    c = np.array(c0, dtype=np.complex128)
    r = f - L @ c
    p = L.conj().T @ r
    rr = _norm2(r)
    res = [float(np.sqrt(rr))]
    for _ in range(iters):
        pp = _norm2(p)
        if pp == 0:
            break
        alpha = rr / pp
        c = c + complex(alpha) * p
        r = r - complex(alpha) * (L @ p)
        rr_new = _norm2(r)
        beta = rr_new / rr
        p = L.conj().T @ r + complex(beta) * p
        rr = rr_new
        res.append(float(np.sqrt(rr)))
    return c, res


def midpoint_guess(B, xyz, f, kappa, N):
    """Mid-point rule of the paper's last test: h^3 sum_i f(x_i) conj(H(x_i)) e^{-|x_i|^2}."""
    xyz = np.asarray(xyz, dtype=np.float64).reshape(-1, 3)
    h3 = (2.0 * kappa / N) ** 3
    wts = h3 * np.exp(-np.sum(xyz * xyz, axis=1))
    a, _ = direct.adjoint(B, xyz, wts * f)
    return a


def cartesian_grid(N, kappa):
    """G_N = kappa [2j/N - 1, 2k/N - 1, 2l/N - 1], j, k, l = 0..N-1 (Sect. 8, last test)."""
    t = kappa * (2.0 * np.arange(N) / N - 1.0)
    X, Y, Z = np.meshgrid(t, t, t, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
