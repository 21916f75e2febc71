"""ctypes wrapper of the C direct-summation oracle (``sgl_oracle.c``).

TEST INFRASTRUCTURE ONLY (see the package docstring).  The library is compiled
with gcc on first use (or by ``__graft_entry__.build()``) into ``oracle/_build``.
Two builds exist: ``double`` (the oracle proper) and ``long double`` (the same
source with every step rounded in a wider type; a self-check of rounding).
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sgl_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIBS = {}
_LOCK = threading.Lock()


def build(kind="double", force=False):
    """Compile the oracle with gcc; returns the path of the shared library."""
    os.makedirs(_BUILD, exist_ok=True)
    name = "liboracle_%s.so" % ("ld" if kind == "long double" else "d")
    out = os.path.join(_BUILD, name)
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm", "-lpthread"]
        if kind == "long double":
            cmd.insert(1, "-DORACLE_REAL=long double")
        subprocess.check_call(cmd)
        os.replace(tmp, out)
    return out


def _lib(kind="double"):
    with _LOCK:
        if kind not in _LIBS:
            lib = ctypes.CDLL(build(kind))
            dp = ctypes.POINTER(ctypes.c_double)
            i64 = ctypes.c_int64
            lib.oracle_num_coeffs.restype = i64
            lib.oracle_num_coeffs.argtypes = [ctypes.c_int]
            for f in (lib.oracle_forward, lib.oracle_adjoint):
                f.restype = ctypes.c_int
                f.argtypes = [ctypes.c_int, i64, dp, dp, dp, ctypes.c_int]
            lib.oracle_grad_points.restype = ctypes.c_int
            lib.oracle_grad_points.argtypes = [ctypes.c_int, i64, dp, dp, dp, dp, ctypes.c_int]
            lib.oracle_basis.argtypes = [ctypes.c_int, dp, dp]
            lib.oracle_laguerre.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, dp]
            lib.oracle_radial.argtypes = [ctypes.c_int, ctypes.c_double, dp]
            lib.oracle_legendre.argtypes = [ctypes.c_int, ctypes.c_double, dp]
            lib.oracle_mu.restype = i64
            lib.oracle_mu.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
            ip = ctypes.POINTER(ctypes.c_int)
            lib.oracle_nlm.argtypes = [i64, ip, ip, ip]
            lib.oracle_real_bytes.restype = ctypes.c_int
            _LIBS[kind] = lib
        return _LIBS[kind]


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c128(a, n):
    a = np.ascontiguousarray(a, dtype=np.complex128).reshape(-1)
    assert a.size == n, (a.size, n)
    return a


def num_coeffs(B):
    """B(B+1)(2B+1)/6 coefficients for bandwidth B (Sect. 1)."""
    return int(_lib().oracle_num_coeffs(int(B)))


def forward(B, xyz, coef, nthreads=0, kind="double"):
    """f_i = sum_mu coef_mu H_mu(x_i) (Def. of the NDSGLFT).  Returns (f, threads used)."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    M = xyz.shape[0]
    coef = _c128(coef, num_coeffs(B))
    out = np.zeros(M, dtype=np.complex128)
    t = _lib(kind).oracle_forward(int(B), M, _p(xyz), _p(coef), _p(out), int(nthreads))
    if t < 0:
        raise ValueError("oracle_forward rejected its arguments")
    return out, t


def adjoint(B, xyz, y, nthreads=0, kind="double"):
    """c'_mu = sum_i conj(H_mu(x_i)) y_i (Lambda^H).  Returns (c', threads used)."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    M = xyz.shape[0]
    y = _c128(y, M)
    out = np.zeros(num_coeffs(B), dtype=np.complex128)
    t = _lib(kind).oracle_adjoint(int(B), M, _p(xyz), _p(y), _p(out), int(nthreads))
    if t < 0:
        raise ValueError("oracle_adjoint rejected its arguments")
    return out, t


def grad_points(B, xyz, coef, g, nthreads=0, kind="double"):
    """grad_i = Re(conj(g_i) grad_x f(x_i)) with f = Lambda coef.  Returns ([M,3], threads used)."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    M = xyz.shape[0]
    coef = _c128(coef, num_coeffs(B))
    g = _c128(g, M)
    out = np.zeros((M, 3), dtype=np.float64)
    t = _lib(kind).oracle_grad_points(int(B), M, _p(xyz), _p(coef), _p(g), _p(out), int(nthreads))
    if t < 0:
        raise ValueError("oracle_grad_points rejected its arguments")
    return out, t


def basis(B, x, kind="double"):
    """All H_mu(x), mu = 0..Nc-1, at one point x (3,)."""
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(3)
    out = np.zeros(num_coeffs(B), dtype=np.complex128)
    _lib(kind).oracle_basis(int(B), _p(x), _p(out))
    return out


def laguerre(K, a, x, kind="double"):
    """Generalized Laguerre L_k^{(a)}(x), k = 0..K."""
    out = np.zeros(K + 1)
    _lib(kind).oracle_laguerre(int(K), float(a), float(x), _p(out))
    return out


def radial(B, r, kind="double"):
    """N_nl R_nl(r) as an array [B+1, B] indexed [n, l] (zero where l >= n)."""
    out = np.zeros((B + 1) * B)
    _lib(kind).oracle_radial(int(B), float(r), _p(out))
    return out.reshape(B + 1, B)


def legendre(B, theta, kind="double"):
    """Q_lm P_lm(cos theta) as an array [B, B] indexed [l, m], m >= 0."""
    out = np.zeros(B * B)
    _lib(kind).oracle_legendre(int(B), float(theta), _p(out))
    return out.reshape(B, B)


def mu(n, l, m):
    """Linear coefficient index of (n, l, m) (Sect. 1)."""
    return int(_lib().oracle_mu(int(n), int(l), int(m)))


def nlm(mu_):
    """(n, l, m) of a linear index, by search (the closed form of Sect. 1 is not used)."""
    n, l, m = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _lib().oracle_nlm(int(mu_), ctypes.byref(n), ctypes.byref(l), ctypes.byref(m))
    return n.value, l.value, m.value


def real_bytes(kind="double"):
    return int(_lib(kind).oracle_real_bytes())
