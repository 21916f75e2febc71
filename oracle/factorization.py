"""The paper's exact factorization of Lambda, up to the trigonometric
coefficients eta, written as the steps of Sect. 6 in their order.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Slow and small-B only.

Steps (Sect. 6, "Derivation of the fast algorithms"):
  radial subtransform
    g_lm(r_j) = sum_{n=l+1}^{B} fhat_nlm N_nl R_nl(r_j),  r_j = rho (1 + cos w_j)/2,
                w_j = (2j+1) pi / (4B), j = 0..2B-1
    alpha_{.lm} = D_2B Ctilde_2B [g_lm(r_j)]_j                     (eq. for alpha_{kappa l m})
    beta_{kappa lm} = alpha_0 (kappa=0), alpha_|kappa|/2 (0<|kappa|<2B), 0 (kappa=-2B)
  spherical subtransform, for every kappa0 in I_4B and |m| < B
    h_{kappa0,m}(cos w_j) = sum_{l=|m|}^{B-1} beta_{kappa0 l m} Q_lm P_lm(cos w_j)
    m even: eps = D_2B Ctilde_2B [h(cos w_j)]_j, zeta as alpha -> beta above
    m odd:  eps = D_2B Ctilde_2B V_B [h(cos w_j)]_j, V_B = diag(1/sin w_j),
            zeta_kappa = sgn(kappa)/(4i) * {0 | 2eps_0 - eps_2 | eps_{|k|-1} - eps_{|k|+1} | eps_{|k|-1} | 0}
  eta_k = zeta_{kappa0 kappa1 kappa2} for |kappa2| < B, else 0, k in I^3_4B
  and f(x_i) = sum_k eta_k exp(i <k, xtilde_i>), xtilde = [arccos gamma(r), theta, phi],
  gamma(r) = (2r - rho)/rho.

Readings of the printed text used here: V_B's node uses the 2B-point angle
(2j+1) pi / (4B) (the printed "4n" is read as 4B); Q_{l,-m} P_{l,-m} =
(-1)^m Q_lm P_lm (the Rodrigues formula of Sect. 4 read for negative order).
"""
import numpy as np

from . import direct


def dct_tilde(n):
    """Ctilde_n = D_n C_n, C_n = [cos(i w_j)], w_j = (2j+1) pi / (2n) (Def. of the DCT, Sect. 3)."""
    w = (2 * np.arange(n) + 1) * np.pi / (2 * n)
    C = np.cos(np.outer(np.arange(n), w))
    D = np.diag(np.r_[1.0 / np.sqrt(n), np.full(n - 1, np.sqrt(2.0 / n))])
    return D, D @ C


def chebyshev_to_exponential(a):
    """alpha_0..alpha_{n-1} -> beta_kappa, kappa in I_{2n} (index kappa + n); the map A_B of Sect. 6."""
    n = a.shape[0]
    out = np.zeros((2 * n,) + a.shape[1:], dtype=np.complex128)
    out[n] = a[0]
    for k in range(1, n):
        out[n + k] = a[k] / 2
        out[n - k] = a[k] / 2
    return out  # out[0] is kappa = -n, left zero


def coefficient_cube(B, coef):
    """fhat in mu order -> array C[n, l, m + B - 1] (n = 1..B at index n)."""
    C = np.zeros((B + 1, B, 2 * B - 1), dtype=np.complex128)
    mu = 0
    for n in range(1, B + 1):
        for l in range(n):
            for m in range(-l, l + 1):
                C[n, l, m + B - 1] = coef[mu]
                mu += 1
    return C


def eta(B, coef, rho):
    """Coefficients eta_k, k in I^3_{4B}, as a complex array [4B, 4B, 4B] indexed k + 2B."""
    coef = np.asarray(coef, dtype=np.complex128)
    n2 = 2 * B
    w = (2 * np.arange(n2) + 1) * np.pi / (4 * B)          # w_j, j = 0..2B-1
    D, Ct = dct_tilde(n2)
    DCt = D @ Ct                                            # D_2B Ctilde_2B
    Cf = coefficient_cube(B, coef)
    # radial subtransform
    rj = rho * (1 + np.cos(w)) / 2
    Rad = np.stack([direct.radial(B, r) for r in rj])       # [j, n, l]
    g = np.einsum("jnl,nlm->jlm", Rad, Cf)                 # g_lm(r_j)
    alpha = np.einsum("kj,jlm->klm", DCt, g)               # [kappa, l, m]
    beta = chebyshev_to_exponential(alpha)                  # [kappa0 + 2B, l, m]
    # spherical subtransform
    Lg = np.stack([direct.legendre(B, wj) for wj in w])     # [j, l, |m|] = Q P(cos w_j)
    ms = np.arange(-(B - 1), B)
    QP = np.zeros((n2, B, 2 * B - 1))
    for im, m in enumerate(ms):
        am = abs(m)
        QP[:, :, im] = Lg[:, :, am] * ((-1.0) ** am if m < 0 else 1.0)
    h = np.einsum("alm,jlm->ajm", beta, QP)                # h_{kappa0,m}(cos w_j), [kappa0, j, m]
    zeta = np.zeros((4 * B, 4 * B, 2 * B - 1), dtype=np.complex128)
    V = 1.0 / np.sin(w)
    for im, m in enumerate(ms):
        if m % 2 == 0:
            eps = np.einsum("kj,aj->ka", DCt, h[:, :, im])           # [kappa, kappa0]
            zeta[:, :, im] = chebyshev_to_exponential(eps).T        # [kappa0, kappa1]
        else:
            eps = np.einsum("kj,aj->ka", DCt, h[:, :, im] * V[None, :])
            z = np.zeros((4 * B, 4 * B), dtype=np.complex128)      # [kappa1 + 2B, kappa0]
            for k in range(1, 2 * B):
                if k == 1:
                    v = 2 * eps[0] - eps[2]
                elif k < 2 * B - 2:
                    v = eps[k - 1] - eps[k + 1]
                else:
                    v = eps[k - 1]
                z[2 * B + k] = v / (4j)
                z[2 * B - k] = -v / (4j)
            zeta[:, :, im] = z.T
    out = np.zeros((4 * B, 4 * B, 4 * B), dtype=np.complex128)
    out[:, :, 2 * B - (B - 1): 2 * B + B] = zeta
    return out


def torus_points(xyz, rho):
    """xtilde_i = [arccos gamma(r_i), theta_i, phi_i] in [0, 2 pi)^3 (eq. for the transformed points)."""
    xyz = np.asarray(xyz, dtype=np.float64).reshape(-1, 3)
    r = np.linalg.norm(xyz, axis=1)
    gam = np.clip((2 * r - rho) / rho, -1.0, 1.0)
    theta = np.arctan2(np.hypot(xyz[:, 0], xyz[:, 1]), xyz[:, 2])
    phi = np.mod(np.arctan2(xyz[:, 1], xyz[:, 0]), 2 * np.pi)
    return np.stack([np.arccos(gam), theta, phi], axis=1)


def ndft(eta_cube, t, chunk=64):
    """f_i = sum_{k in I^3_n} eta_k exp(i <k, t_i>) (the NDFT of Sect. 2), cube indexed k + n/2."""
    n0, n1, n2 = eta_cube.shape
    k0 = np.arange(n0) - n0 // 2
    k1 = np.arange(n1) - n1 // 2
    k2 = np.arange(n2) - n2 // 2
    t = np.asarray(t, dtype=np.float64).reshape(-1, 3)
    out = np.zeros(t.shape[0], dtype=np.complex128)
    flat = eta_cube.reshape(n0 * n1, n2)
    for s in range(0, t.shape[0], chunk):
        tt = t[s:s + chunk]
        E0 = np.exp(1j * np.outer(tt[:, 0], k0))
        E1 = np.exp(1j * np.outer(tt[:, 1], k1))
        E2 = np.exp(1j * np.outer(tt[:, 2], k2))
        T1 = (flat @ E2.T).reshape(n0, n1, -1)
        T2 = np.einsum("abi,ib->ai", T1, E1)
        out[s:s + chunk] = np.einsum("ai,ia->i", T2, E0)
    return out
