"""The d = 3 NFFT of Sect. 2 with per-dimension grid sizes, and its Gaussian error bound.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Slow and small-size only.

Steps, in the order of Sect. 2:
  1. beta_k = omega_k / phitilde_k for k in I_n, zero on I_{sigma n} minus I_n
  2. alpha = (sigma n)^{-d} F^H beta            (an inverse FFT; numpy's ifftn)
  3. s(t) = sum over l with |sigma n t / 2pi - l| <= q of alpha_l psitilde(t - 2 pi l / sigma n)
with phitilde_k = (2pi)^{-d} int phi(x) exp(-i<k,x>) dx (Poisson summation, Sect. 2).

Windows (per dimension j, grid size N_j = sigma n_j, u = N_j xi / (2 pi)):
  gauss: phi_j(xi) = (2 pi lam)^{-1/2} (N_j / 2pi) exp(-u^2 / (2 lam)),
         lam = sigma q / ((2 sigma - 1) pi); int phi_j exp(-i kappa xi) = exp(-2 lam (pi kappa / N_j)^2)
         (Def. of the Gaussian ansatz, Lemma on its Fourier transform)
  kb:    phi_j(xi) = (N_j / 2pi) (1/pi) sinh(b sqrt(q^2 - u^2)) / sqrt(q^2 - u^2), b = pi (2 - 1/sigma),
         int phi_j exp(-i kappa xi) = I_0(q sqrt(b^2 - (2 pi kappa / N_j)^2))
         (the Kaiser-Bessel pair of the NFFT literature; not in the paper)
"""
import math

import numpy as np
from scipy.special import i0


def gauss_lambda(sigma, q):
    return sigma * q / ((2 * sigma - 1) * math.pi)


def kb_shape(sigma):
    return math.pi * (2.0 - 1.0 / sigma)


def window_fourier(kappa, N, sigma, q, window):
    """int phi_j(xi) exp(-i kappa xi) d xi for the 1-D factor of the window."""
    kappa = np.asarray(kappa, dtype=np.float64)
    if window == "gauss":
        lam = gauss_lambda(sigma, q)
        return np.exp(-2 * lam * (math.pi * kappa / N) ** 2)
    if window == "kb":
        b = kb_shape(sigma)
        w = 2 * math.pi * kappa / N
        arg = np.sqrt(np.maximum(b * b - w * w, 0.0))
        return i0(q * arg)
    raise ValueError(window)


def window_value(xi, N, sigma, q, window):
    """phi_j(xi), truncated to |u| <= q (i.e. psi_j), u = N xi / (2 pi)."""
    u = N * np.asarray(xi, dtype=np.float64) / (2 * math.pi)
    inside = np.abs(u) <= q
    if window == "gauss":
        lam = gauss_lambda(sigma, q)
        v = (N / (2 * math.pi)) / math.sqrt(2 * math.pi * lam) * np.exp(-u * u / (2 * lam))
    elif window == "kb":
        b = kb_shape(sigma)
        s = np.sqrt(np.maximum(q * q - u * u, 0.0))
        with np.errstate(invalid="ignore", divide="ignore"):
            core = np.where(s > 1e-12, np.sinh(b * s) / np.where(s > 1e-12, s, 1.0), b)
        v = (N / (2 * math.pi)) * core / math.pi
    else:
        raise ValueError(window)
    return np.where(inside, v, 0.0)


def nfft(omega, t, sigma, q, window="kb", chunk=256):
    """Approximate p(t_i) = sum_{k in I_n} omega_k exp(i<k,t_i>); omega indexed k + n/2 per axis."""
    n = omega.shape
    N = tuple(int(round(sigma * nj)) for nj in n)
    # 1. deconvolution and zero padding; frequency k sits at index k mod N
    beta = np.zeros(N, dtype=np.complex128)
    ks = [np.arange(nj) - nj // 2 for nj in n]
    phit = [window_fourier(ks[j], N[j], sigma, q, window) / (2 * math.pi) for j in range(3)]
    scaled = omega / (phit[0][:, None, None] * phit[1][None, :, None] * phit[2][None, None, :])
    beta[np.ix_(ks[0] % N[0], ks[1] % N[1], ks[2] % N[2])] = scaled
    # 2. alpha = (sigma n)^{-d} F^H beta
    alpha = np.fft.ifftn(beta)
    # 3. windowed sum over the 2q+1 candidate grid indices per dimension
    t = np.asarray(t, dtype=np.float64).reshape(-1, 3)
    out = np.zeros(t.shape[0], dtype=np.complex128)
    offs = np.arange(-q, q + 1)
    for s in range(0, t.shape[0], chunk):
        tt = t[s:s + chunk]
        idx, wts = [], []
        for j in range(3):
            u = N[j] * tt[:, j] / (2 * math.pi)
            l = np.floor(u)[:, None].astype(np.int64) + offs[None, :]     # candidates around u
            l = np.concatenate([l, (np.floor(u)[:, None] + q + 1).astype(np.int64)], axis=1)
            wts.append(window_value(tt[:, j:j + 1] - 2 * math.pi * l / N[j], N[j], sigma, q, window))
            idx.append(np.mod(l, N[j]))
        vals = alpha[idx[0][:, :, None, None], idx[1][:, None, :, None], idx[2][:, None, None, :]]
        w = wts[0][:, :, None, None] * wts[1][:, None, :, None] * wts[2][:, None, None, :]
        out[s:s + chunk] = np.sum(vals * w, axis=(1, 2, 3))
    return out


def gauss_error_bound(d, sigma, q):
    """Factor C with E_inf <= C ||w||_1 for the Gaussian window (Thm. on the d-dim. NFFT error).

    Valid for sigma >= (sqrt(d) + 1) / 2 and lambda = sigma q / ((2 sigma - 1) pi).
    """
    if sigma < (math.sqrt(d) + 1) / 2:
        raise ValueError("bound needs sigma >= (sqrt(d)+1)/2")
    a = (2 ** d - 1) * (2 + 1 / (math.pi * q)) ** d
    b = (3 ** d - 1) / q ** (d / 2) * (math.sqrt((2 * sigma - 1) / (2 * sigma)) + math.sqrt(2 * sigma / (2 * sigma - 1)) / (2 * math.pi)) ** d
    e = math.exp(-q * math.pi * (1 - (1 + d / (2 * sigma - 1)) / (2 * sigma)))
    return (a + b) * e


def fft_size(target):
    """Smallest even 2-3-5-smooth integer >= target (the plan's oversampled grid sizes)."""
    n = math.ceil(target - 1e-9)
    n += n % 2
    while True:
        m = n
        for f in (2, 3, 5):
            while m % f == 0:
                m //= f
        if m == 1:
            return n
        n += 2


def single_frequency_error(N, n, K, q, window, nfrac=128):
    """max over |k| <= K and t = 2 pi (l0 + f) / N, f = (i + 1/2) / nfrac, of |e^{ikt} - s(t)|, where
    s is the 1-D NFFT of Sect. 2 (steps 1-3) applied to the single coefficient omega_k = 1 on a grid
    of N = sigma n points (sigma = N / n).  By translation invariance l0 = 0 suffices."""
    sigma = N / n
    ks = np.arange(-K, K + 1)
    phit = window_fourier(ks, N, sigma, q, window) / (2 * math.pi)              # step 1: beta_k = 1 / phitilde_k
    f = (np.arange(nfrac) + 0.5) / nfrac
    t = 2 * math.pi * f / N
    ls = np.arange(-q, q + 2)                                                    # every l with |N t / 2 pi - l| <= q
    # step 2: alpha_l = N^{-1} beta_k e^{2 pi i k l / N};  step 3: s(t) = sum_l alpha_l phi(t - 2 pi l / N)
    wts = window_value(t[:, None] - 2 * math.pi * ls[None, :] / N, N, sigma, q, window)           # [f, l]
    ph = np.exp(2j * math.pi * ks[:, None] * ls[None, :] / N)                                     # [k, l]
    s = (ph @ wts.T) / (N * phit[:, None])                                                        # [k, f]
    exact = np.exp(1j * ks[:, None] * t[None, :])
    return float(np.abs(exact - s).max())


def sgl_nfft_bound(B, q, sigma, window):
    """Error bound of the NFSGLFT per unit ||eta||_1: the three axes' single-frequency errors
    combined as prod (1 + e_d) - 1 (|a b c - a' b' c'| <= prod (1 + e_d) - 1 for |a| = |b| = |c| = 1,
    |a - a'| <= e_0, ...), on the axes n = (4B, 2B, 2B), |k| <= (2B - 2, B - 1, B - 1) of Sect. 6."""
    n = (4 * B, 2 * B, 2 * B)
    K = (2 * B - 2, B - 1, B - 1)
    b = 1.0
    for d in range(3):
        b *= 1.0 + single_frequency_error(fft_size(sigma * n[d]), n[d], K[d], q, window)
    return b - 1.0
