"""Thin ctypes binding of libsgl.so (include/sgl.h): argument marshalling only.

Every transform step runs in the library's CUDA kernels.  PyTorch supplies the
device memory and the stream: tensors are passed by ``data_ptr()`` and calls are
issued on ``torch.cuda.current_stream()``.  There is no CPU fallback: without the
library (or without a GPU) every call raises :class:`SGLError`.
"""
import ctypes
import os
import threading

import torch

from . import build as _build

PREC_FP64, PREC_FP32_MIXED = 0, 1
WIN_KB, WIN_GAUSS = 0, 1
FLAG_HOST_IO, FLAG_PROFILE, FLAG_SIMT, FLAG_TC, FLAG_NATIVE_FP64, FLAG_OVERLAP_POINTS = 1, 2, 4, 8, 16, 32
FLAG_GENERIC_FFT = 64
FLAG_FULL_GRID = 128
NUM_STAGES = 12

_STATUS = {0: "SGL_OK", 1: "SGL_ERR_ARG", 2: "SGL_ERR_ALLOC", 3: "SGL_ERR_CUDA", 4: "SGL_ERR_NONFINITE",
           5: "SGL_ERR_TIMEOUT", 6: "SGL_ERR_UNSUPPORTED", 7: "SGL_ERR_STATE"}

_LIB = None
_LOCK = threading.Lock()


class SGLError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_STATUS.get(status, status), msg))
        self.status = status


class PlanInfo(ctypes.Structure):
    _fields_ = [("B", ctypes.c_int), ("q", ctypes.c_int), ("precision", ctypes.c_int), ("window", ctypes.c_int),
                ("num_coeffs", ctypes.c_int64), ("M_max", ctypes.c_int64), ("M", ctypes.c_int64),
                ("n", ctypes.c_int * 3), ("N", ctypes.c_int * 3), ("rows", ctypes.c_int * 3),
                ("sigma_eff", ctypes.c_double * 3), ("workspace_bytes", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("tensor_cores", ctypes.c_int), ("sym_grid", ctypes.c_int)]


def library_path():
    return _build.LIB


def load_library(build_if_missing=True):
    """Load libsgl.so (building it in-tree first if it is missing and nvcc exists)."""
    global _LIB
    with _LOCK:
        if _LIB is not None:
            return _LIB
        path = library_path()
        if not os.path.exists(path):
            if not build_if_missing:
                raise SGLError(3, "libsgl.so is not built (%s)" % path)
            _build.build()
        lib = ctypes.CDLL(path)
        vp, dp, i64 = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int64
        lib.sgl_num_coeffs.restype = i64
        lib.sgl_num_coeffs.argtypes = [ctypes.c_int]
        lib.sgl_last_error.restype = ctypes.c_char_p
        lib.sgl_plan_create.restype = ctypes.c_int
        lib.sgl_plan_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, i64, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_double, ctypes.c_uint, vp]
        lib.sgl_plan_destroy.restype = None
        lib.sgl_plan_destroy.argtypes = [vp]
        for name, args in [("sgl_set_stream", [vp, vp]), ("sgl_plan_info", [vp, ctypes.POINTER(PlanInfo)]),
                           ("sgl_set_points", [vp, vp, i64]), ("sgl_get_rho", [vp, dp]),
                           ("sgl_forward", [vp, vp, vp]), ("sgl_adjoint", [vp, vp, vp]),
                           ("sgl_grad_points", [vp, vp, vp, vp]), ("sgl_trig_coeffs", [vp, vp, vp]),
                           ("sgl_forward_host", [vp, vp, i64, vp, vp]), ("sgl_adjoint_host", [vp, vp, i64, vp, vp]),
                           ("sgl_grad_points_host", [vp, vp, i64, vp, vp, vp]),
                           ("sgl_forward_grad", [vp, vp, vp, vp, vp]),
                           ("sgl_inverse", [vp, vp, vp, ctypes.c_int, ctypes.c_double, ctypes.c_int, dp,
                                            ctypes.POINTER(ctypes.c_int)]),
                           ("sgl_midpoint_guess", [vp, vp, vp, vp]),
                           ("sgl_nfft_error_bound", [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, dp]),
                           ("sgl_plan_error_bound", [vp, dp]),
                           ("sgl_choose_cutoff", [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                                  ctypes.POINTER(ctypes.c_int)]),
                           ("sgl_eta_l1", [vp, vp, dp]),
                           ("sgl_test_hooks", [vp, ctypes.c_uint, i64]), ("sgl_test_fail_alloc", [ctypes.c_int]),
                           ("sgl_choose_params", [ctypes.c_int, i64, ctypes.c_int, ctypes.c_int, ctypes.c_double, dp,
                                                  ctypes.POINTER(ctypes.c_int), dp]),
                           ("sgl_forward_grad_host", [vp, vp, i64, vp, vp, vp, vp]),
                           ("sgl_profile", [vp, dp, ctypes.POINTER(i64)]), ("sgl_sync", [vp]),
                           ("sgl_trig_coeffs_noalloc", [ctypes.c_int, vp, i64, vp, vp, vp])]:
            f = getattr(lib, name)
            f.restype = ctypes.c_int
            f.argtypes = args
        pp = ctypes.POINTER(ctypes.c_void_p)
        lib.sgl_batch_create.restype = ctypes.c_int
        lib.sgl_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(i64), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_uint, vp]
        lib.sgl_batch_destroy.restype = None
        lib.sgl_batch_destroy.argtypes = [vp]
        for name, args in [("sgl_batch_use_graph", [vp, ctypes.c_int]), ("sgl_batch_set_points", [vp, pp, ctypes.POINTER(i64)]),
                           ("sgl_batch_forward", [vp, pp, pp]), ("sgl_batch_adjoint", [vp, pp, pp]),
                           ("sgl_batch_info", [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(i64), ctypes.POINTER(i64)]),
                           ("sgl_batch_sync", [vp]), ("sgl_batch_set_lanes", [vp, ctypes.c_int]),
                           ("sgl_batch_lanes", [vp, ctypes.POINTER(ctypes.c_int)]),
                           ("sgl_batch_autotune", [vp, ctypes.c_char_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)])]:
            f = getattr(lib, name)
            f.restype = ctypes.c_int
            f.argtypes = args
        lib.sgl_noalloc_max_b.restype = ctypes.c_int
        lib.sgl_noalloc_max_b.argtypes = []
        lib.sgl_stage_name.restype = ctypes.c_char_p
        lib.sgl_stage_name.argtypes = [ctypes.c_int]
        _LIB = lib
        return lib


def _check(st):
    if st != 0:
        raise SGLError(st, _LIB.sgl_last_error().decode())


def num_coeffs(B):
    return int(load_library().sgl_num_coeffs(int(B)))


def nfft_error_bound(B, window=WIN_KB, q=8, sigma=2.0):
    """sgl_nfft_error_bound: max |f - f~| <= bound * ||eta||_1 for a plan of these parameters."""
    b = ctypes.c_double()
    _check(load_library().sgl_nfft_error_bound(int(B), int(window), int(q), float(sigma), ctypes.byref(b)))
    return b.value


def choose_cutoff(B, tol, window=WIN_KB, sigma=2.0):
    """sgl_choose_cutoff: the smallest q whose bound per unit ||eta||_1 is <= tol."""
    q = ctypes.c_int()
    _check(load_library().sgl_choose_cutoff(int(B), int(window), float(sigma), float(tol), ctypes.byref(q)))
    return q.value


def choose_params(B, M, tol, precision=PREC_FP64, window=WIN_KB):
    """sgl_choose_params: (sigma, q, model_ms) -- the cheapest pair (by the GB300 cost model) whose
    bound per unit ||eta||_1 is <= tol."""
    sg, q, ms = ctypes.c_double(), ctypes.c_int(), ctypes.c_double()
    _check(load_library().sgl_choose_params(int(B), int(M), int(precision), int(window), float(tol), ctypes.byref(sg),
                                            ctypes.byref(q), ctypes.byref(ms)))
    return sg.value, q.value, ms.value


def _stream_handle(device):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _dev_tensor(t, dtype, shape, name, device):
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch.Tensor" % name)
    if t.device.type != "cuda" or t.device != device:
        raise ValueError("%s must live on %s" % (name, device))
    if t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if tuple(t.shape) != tuple(shape):
        raise ValueError("%s must have shape %s, got %s" % (name, tuple(shape), tuple(t.shape)))
    return t.contiguous()


class Plan:
    """One NFSGLFT plan (sgl_plan_create): bandwidth B, up to M_max points."""

    def __init__(self, B, M_max, precision=PREC_FP64, window=WIN_KB, q=8, sigma=2.0, host_io=False, profile=False,
                 device=None, simt=False, tensor_cores=False, native_fp64=False, overlap_points=False,
                 generic_fft=False, full_grid=False):
        if not torch.cuda.is_available():
            raise SGLError(3, "no CUDA device: the NFSGLFT runs only on the GPU")
        self.lib = load_library()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else torch.device(device).index or 0)
        self.B, self.M_max = int(B), int(M_max)
        self.precision, self.window, self.q, self.sigma = int(precision), int(window), int(q), float(sigma)
        self._h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            st = self.lib.sgl_plan_create(ctypes.byref(self._h), self.B, self.M_max, self.precision, self.window,
                                          self.q, self.sigma,
                                          (FLAG_HOST_IO if host_io else 0) | (FLAG_PROFILE if profile else 0) | (FLAG_SIMT if simt else 0)
                                          | (FLAG_TC if tensor_cores else 0) | (FLAG_NATIVE_FP64 if native_fp64 else 0)
                                          | (FLAG_OVERLAP_POINTS if overlap_points else 0)
                                          | (FLAG_GENERIC_FFT if generic_fft else 0)
                                          | (FLAG_FULL_GRID if full_grid else 0),
                                          _stream_handle(self.device))
        _check(st)
        self.Nc = num_coeffs(self.B)
        self.M = 0
        self._xyz = None

    def close(self):
        if self._h:
            self.lib.sgl_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _stream(self):
        _check(self.lib.sgl_set_stream(self._h, _stream_handle(self.device)))

    def info(self):
        inf = PlanInfo()
        _check(self.lib.sgl_plan_info(self._h, ctypes.byref(inf)))
        return {"B": inf.B, "q": inf.q, "precision": inf.precision, "window": inf.window,
                "num_coeffs": inf.num_coeffs, "M_max": inf.M_max, "M": inf.M, "n": list(inf.n), "N": list(inf.N),
                "rows": list(inf.rows), "sigma_eff": list(inf.sigma_eff), "workspace_bytes": inf.workspace_bytes,
                "kernel_launches": inf.kernel_launches,
                "tensor_cores": {"interp": bool(inf.tensor_cores & 1), "grad": bool(inf.tensor_cores & 2),
                                 "spread": bool(inf.tensor_cores & 4)},
                "sym_grid": bool(inf.sym_grid)}

    def profile(self):
        """{stage: (milliseconds, timed calls)} since the last call (plan made with profile=True)."""
        ms = (ctypes.c_double * NUM_STAGES)()
        cnt = (ctypes.c_int64 * NUM_STAGES)()
        _check(self.lib.sgl_profile(self._h, ms, cnt))
        return {self.lib.sgl_stage_name(i).decode(): (ms[i], cnt[i]) for i in range(NUM_STAGES)}

    def set_points(self, xyz):
        xyz = _dev_tensor(xyz, torch.float64, (xyz.shape[0], 3), "xyz", self.device)
        self._stream()
        _check(self.lib.sgl_set_points(self._h, ctypes.c_void_p(xyz.data_ptr()), xyz.shape[0]))
        self.M = xyz.shape[0]
        self._xyz = xyz            # keep alive until the stream has consumed it
        return self

    def rho(self):
        v = ctypes.c_double()
        _check(self.lib.sgl_get_rho(self._h, ctypes.byref(v)))
        return v.value

    def forward(self, coef, out=None):
        coef = _dev_tensor(coef, torch.complex128, (self.Nc,), "coef", self.device)
        if out is None:
            out = torch.empty(self.M, dtype=torch.complex128, device=self.device)
        out = _dev_tensor(out, torch.complex128, (self.M,), "out", self.device)
        self._stream()
        _check(self.lib.sgl_forward(self._h, ctypes.c_void_p(coef.data_ptr()), ctypes.c_void_p(out.data_ptr())))
        return out

    def adjoint(self, vals, out=None):
        vals = _dev_tensor(vals, torch.complex128, (self.M,), "vals", self.device)
        if out is None:
            out = torch.empty(self.Nc, dtype=torch.complex128, device=self.device)
        out = _dev_tensor(out, torch.complex128, (self.Nc,), "out", self.device)
        self._stream()
        _check(self.lib.sgl_adjoint(self._h, ctypes.c_void_p(vals.data_ptr()), ctypes.c_void_p(out.data_ptr())))
        return out

    def grad_points(self, coef, gout, out=None):
        coef = _dev_tensor(coef, torch.complex128, (self.Nc,), "coef", self.device)
        gout = _dev_tensor(gout, torch.complex128, (self.M,), "gout", self.device)
        if out is None:
            out = torch.empty((self.M, 3), dtype=torch.float64, device=self.device)
        out = _dev_tensor(out, torch.float64, (self.M, 3), "out", self.device)
        self._stream()
        _check(self.lib.sgl_grad_points(self._h, ctypes.c_void_p(coef.data_ptr()), ctypes.c_void_p(gout.data_ptr()),
                                        ctypes.c_void_p(out.data_ptr())))
        return out

    def forward_grad(self, coef, gout, vals=None, gxyz=None):
        """(f = Lambda coef, Re(conj(gout) grad_x f)) from one conversion, FFT and windowed sweep."""
        coef = _dev_tensor(coef, torch.complex128, (self.Nc,), "coef", self.device)
        gout = _dev_tensor(gout, torch.complex128, (self.M,), "gout", self.device)
        if vals is None:
            vals = torch.empty(self.M, dtype=torch.complex128, device=self.device)
        if gxyz is None:
            gxyz = torch.empty((self.M, 3), dtype=torch.float64, device=self.device)
        vals = _dev_tensor(vals, torch.complex128, (self.M,), "vals", self.device)
        gxyz = _dev_tensor(gxyz, torch.float64, (self.M, 3), "gxyz", self.device)
        self._stream()
        _check(self.lib.sgl_forward_grad(self._h, ctypes.c_void_p(coef.data_ptr()), ctypes.c_void_p(gout.data_ptr()),
                                         ctypes.c_void_p(vals.data_ptr()), ctypes.c_void_p(gxyz.data_ptr())))
        return vals, gxyz

    def inverse(self, vals, coef0=None, iters=100, tol=0.0, method="auto"):
        """iNFSGLFT: coefficients from samples at the plan's points by CGNR / CGNE.
        Returns (coef, relative residual ||f - Lambda c|| / ||f||, iterations done)."""
        vals = _dev_tensor(vals, torch.complex128, (self.M,), "vals", self.device)
        coef = (torch.zeros(self.Nc, dtype=torch.complex128, device=self.device) if coef0 is None else
                _dev_tensor(coef0, torch.complex128, (self.Nc,), "coef0", self.device).clone())
        m = {"auto": 0, "cgnr": 1, "cgne": 2}[method]
        res = ctypes.c_double(0.0)
        done = ctypes.c_int(0)
        self._stream()
        _check(self.lib.sgl_inverse(self._h, ctypes.c_void_p(vals.data_ptr()), ctypes.c_void_p(coef.data_ptr()), int(iters),
                                    float(tol), m, ctypes.byref(res), ctypes.byref(done)))
        return coef, res.value, done.value

    def error_bound(self):
        """sgl_plan_error_bound: max |f - f~| <= error_bound() * eta_l1(coef)."""
        b = ctypes.c_double()
        _check(self.lib.sgl_plan_error_bound(self._h, ctypes.byref(b)))
        return b.value

    def eta_l1(self, coef):
        """sgl_eta_l1: ||eta||_1 of the trigonometric coefficients of coef at the current points."""
        coef = _dev_tensor(coef, torch.complex128, (self.Nc,), "coef", self.device)
        v = ctypes.c_double()
        self._stream()
        _check(self.lib.sgl_eta_l1(self._h, ctypes.c_void_p(coef.data_ptr()), ctypes.byref(v)))
        return v.value

    def midpoint_guess(self, vals, weights):
        """Lambda^H (weights * vals): the quadrature initial guess of the inverse transform."""
        vals = _dev_tensor(vals, torch.complex128, (self.M,), "vals", self.device)
        weights = _dev_tensor(weights, torch.float64, (self.M,), "weights", self.device)
        out = torch.empty(self.Nc, dtype=torch.complex128, device=self.device)
        self._stream()
        _check(self.lib.sgl_midpoint_guess(self._h, ctypes.c_void_p(vals.data_ptr()), ctypes.c_void_p(weights.data_ptr()),
                                           ctypes.c_void_p(out.data_ptr())))
        return out

    def trig_coeffs(self, coef):
        """eta_k on |k0| <= 2B-2, |k1|, |k2| <= B-1 as complex128 [4B-3, 2B-1, 2B-1]."""
        coef = _dev_tensor(coef, torch.complex128, (self.Nc,), "coef", self.device)
        B = self.B
        out = torch.empty((4 * B - 3, 2 * B - 1, 2 * B - 1), dtype=torch.complex128, device=self.device)
        self._stream()
        _check(self.lib.sgl_trig_coeffs(self._h, ctypes.c_void_p(coef.data_ptr()), ctypes.c_void_p(out.data_ptr())))
        return out

    # Host-buffer calls: numpy or pinned-CPU-tensor buffers, copies inside the call, synchronous.
    # xyz_host None keeps the points of the previous call (no copy, no re-binning).
    def _pts(self, xyz_host):
        if xyz_host is None:
            return None, self.M
        return _host_ptr(xyz_host), int(xyz_host.shape[0])

    def forward_host(self, xyz_host, coef_host, vals_host):
        px, m = self._pts(xyz_host)
        _check(self.lib.sgl_forward_host(self._h, px, m, _host_ptr(coef_host), _host_ptr(vals_host)))
        self.M = m
        return vals_host

    def adjoint_host(self, xyz_host, vals_host, coef_host):
        px, m = self._pts(xyz_host)
        _check(self.lib.sgl_adjoint_host(self._h, px, m, _host_ptr(vals_host), _host_ptr(coef_host)))
        self.M = m
        return coef_host

    def grad_points_host(self, xyz_host, coef_host, gout_host, gxyz_host):
        px, m = self._pts(xyz_host)
        _check(self.lib.sgl_grad_points_host(self._h, px, m, _host_ptr(coef_host), _host_ptr(gout_host), _host_ptr(gxyz_host)))
        self.M = m
        return gxyz_host

    def forward_grad_host(self, xyz_host, coef_host, gout_host, vals_host, gxyz_host):
        px, m = self._pts(xyz_host)
        _check(self.lib.sgl_forward_grad_host(self._h, px, m, _host_ptr(coef_host), _host_ptr(gout_host), _host_ptr(vals_host),
                                              _host_ptr(gxyz_host)))
        self.M = m
        return vals_host, gxyz_host

    def sync(self):
        _check(self.lib.sgl_sync(self._h))


class BatchPlan:
    """Many independent transforms issued together (sgl_batch_*): instance i has bandwidth
    Bs[i] and at most M_maxs[i] points; optional CUDA-graph capture of whole batch calls."""

    def __init__(self, Bs, M_maxs, precision=PREC_FP64, window=WIN_KB, q=8, sigma=2.0, device=None, simt=False,
                 tensor_cores=False, native_fp64=False):
        if not torch.cuda.is_available():
            raise SGLError(3, "no CUDA device: the NFSGLFT runs only on the GPU")
        self.lib = load_library()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else torch.device(device).index or 0)
        self.Bs = [int(b) for b in Bs]
        self.n = len(self.Bs)
        M_maxs = [int(m) for m in M_maxs]
        self._h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            st = self.lib.sgl_batch_create(ctypes.byref(self._h), self.n, (ctypes.c_int * self.n)(*self.Bs),
                                           (ctypes.c_int64 * self.n)(*M_maxs), int(precision), int(window), int(q),
                                           float(sigma), (FLAG_SIMT if simt else 0) | (FLAG_TC if tensor_cores else 0)
                                           | (FLAG_NATIVE_FP64 if native_fp64 else 0),
                                           _stream_handle(self.device))
        _check(st)
        self.Ms = [0] * self.n
        self._keep = []

    def close(self):
        if self._h:
            self.lib.sgl_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def use_graph(self, enable=True):
        _check(self.lib.sgl_batch_use_graph(self._h, 1 if enable else 0))

    def _ptrs(self, tensors):
        return (ctypes.c_void_p * self.n)(*[t.data_ptr() for t in tensors])

    def set_points(self, xyz_list):
        xs = [_dev_tensor(x, torch.float64, (x.shape[0], 3), "xyz", self.device) for x in xyz_list]
        Ms = [x.shape[0] for x in xs]
        _check(self.lib.sgl_batch_set_points(self._h, self._ptrs(xs), (ctypes.c_int64 * self.n)(*Ms)))
        self.Ms = Ms
        self._keep = xs

    def forward(self, coef_list, out_list=None):
        cs = [_dev_tensor(c, torch.complex128, (num_coeffs(B),), "coef", self.device) for c, B in zip(coef_list, self.Bs)]
        if out_list is None:
            out_list = [torch.empty(M, dtype=torch.complex128, device=self.device) for M in self.Ms]
        _check(self.lib.sgl_batch_forward(self._h, self._ptrs(cs), self._ptrs(out_list)))
        return out_list

    def adjoint(self, vals_list, out_list=None):
        vs = [_dev_tensor(v, torch.complex128, (M,), "vals", self.device) for v, M in zip(vals_list, self.Ms)]
        if out_list is None:
            out_list = [torch.empty(num_coeffs(B), dtype=torch.complex128, device=self.device) for B in self.Bs]
        _check(self.lib.sgl_batch_adjoint(self._h, self._ptrs(vs), self._ptrs(out_list)))
        return out_list

    def info(self):
        n, gl, wb = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int64()
        _check(self.lib.sgl_batch_info(self._h, ctypes.byref(n), ctypes.byref(gl), ctypes.byref(wb)))
        return {"n": n.value, "graph_launches": gl.value, "workspace_bytes": wb.value}

    def sync(self):
        _check(self.lib.sgl_batch_sync(self._h))

    def set_lanes(self, lanes):
        _check(self.lib.sgl_batch_set_lanes(self._h, int(lanes)))

    def lanes(self):
        v = ctypes.c_int()
        _check(self.lib.sgl_batch_lanes(self._h, ctypes.byref(v)))
        return v.value

    def autotune(self, cache_path=None):
        """sgl_batch_autotune: (lanes, ms per forward + adjoint, or -1 when taken from the cache)."""
        L, ms = ctypes.c_int(), ctypes.c_double()
        _check(self.lib.sgl_batch_autotune(self._h, cache_path.encode() if cache_path else None, ctypes.byref(L),
                                           ctypes.byref(ms)))
        return L.value, ms.value


def noalloc_max_b():
    """The largest B sgl_trig_coeffs_noalloc accepts (its static scratch limit), from the library."""
    return int(load_library().sgl_noalloc_max_b())


def trig_coeffs_noalloc(B, xyz, coef, out=None):
    """eta for points xyz and coefficients coef without any device allocation by the library
    (sgl_trig_coeffs_noalloc; B <= noalloc_max_b()).  Tensors on the current CUDA device; the
    output tensor may be passed in so that no allocation happens on this side either."""
    lib = load_library()
    dev = xyz.device
    xyz = _dev_tensor(xyz, torch.float64, (xyz.shape[0], 3), "xyz", dev)
    coef = _dev_tensor(coef, torch.complex128, (num_coeffs(B),), "coef", dev)
    if out is None:
        out = torch.empty((4 * B - 3, 2 * B - 1, 2 * B - 1), dtype=torch.complex128, device=dev)
    out = _dev_tensor(out, torch.complex128, (4 * B - 3, 2 * B - 1, 2 * B - 1), "out", dev)
    with torch.cuda.device(dev):
        _check(lib.sgl_trig_coeffs_noalloc(int(B), ctypes.c_void_p(xyz.data_ptr()), xyz.shape[0],
                                           ctypes.c_void_p(coef.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                           _stream_handle(dev)))
    return out


def _host_ptr(a):
    if isinstance(a, torch.Tensor):
        if a.device.type != "cpu" or not a.is_contiguous():
            raise ValueError("host buffers must be contiguous CPU tensors")
        return ctypes.c_void_p(a.data_ptr())
    import numpy as np
    if not isinstance(a, np.ndarray) or not a.flags["C_CONTIGUOUS"]:
        raise ValueError("host buffers must be C-contiguous numpy arrays or CPU tensors")
    return ctypes.c_void_p(a.ctypes.data)
