"""Host-side checks of the C-ABI library (no GPU needed): it loads, exports every
function include/sgl.h declares, and rejects bad arguments before touching CUDA."""
import ctypes
import os
import re

import pytest

import paper_1809_10786_gb300 as sgl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sgl.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sgl_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    return sgl.load_library()


def test_header_declares_the_documented_entry_points():
    names = declared_functions()
    for must in ("sgl_plan_create", "sgl_plan_destroy", "sgl_set_points", "sgl_forward", "sgl_adjoint",
                 "sgl_grad_points", "sgl_num_coeffs", "sgl_last_error"):
        assert must in names


def test_library_exports_every_declared_function(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_num_coeffs(lib):
    for B in (1, 2, 8, 32, 64, 128):
        assert lib.sgl_num_coeffs(B) == B * (B + 1) * (2 * B + 1) // 6
    assert lib.sgl_num_coeffs(0) == -1


@pytest.mark.parametrize("args,word", [
    ((0, 10, 0, 0, 8, 2.0), "B"),
    ((129, 10, 0, 0, 8, 2.0), "B"),
    ((8, -1, 0, 0, 8, 2.0), "M_max"),
    ((8, 10, 2, 0, 8, 2.0), "precision"),
    ((8, 10, 0, 5, 8, 2.0), "window"),
    ((8, 10, 0, 0, 0, 2.0), "q"),
    ((8, 10, 0, 0, 17, 2.0), "q"),
    ((8, 10, 0, 0, 8, 1.2), "sigma"),
    ((8, 10, 0, 0, 8, float("nan")), "sigma"),
])
def test_plan_create_rejects_bad_arguments_without_cuda(lib, args, word):
    h = ctypes.c_void_p(123)
    st = lib.sgl_plan_create(ctypes.byref(h), *args, 0, None)
    assert st == 1                      # SGL_ERR_ARG
    assert h.value is None              # *out cleared
    assert word in lib.sgl_last_error().decode()


@pytest.mark.parametrize("flags,word", [(256, "flag"), (1 << 31, "flag"), (4 | 8, "SGL_FLAG_SIMT")])
def test_plan_create_rejects_bad_flags_without_cuda(lib, flags, word):
    h = ctypes.c_void_p(123)
    st = lib.sgl_plan_create(ctypes.byref(h), 8, 10, 1, 0, 8, 2.0, flags, None)
    assert st == 1
    assert h.value is None
    assert word in lib.sgl_last_error().decode()


def test_null_plan_is_rejected(lib):
    assert lib.sgl_forward(None, None, None) == 1
    assert lib.sgl_set_points(None, None, 0) == 1
    assert lib.sgl_sync(None) == 1
    lib.sgl_plan_destroy(None)          # no-op


def test_out_pointer_required(lib):
    assert lib.sgl_plan_create(None, 8, 10, 0, 0, 8, 2.0, 0, None) == 1


def test_batch_create_rejects_bad_arguments_without_cuda(lib):
    h = ctypes.c_void_p(5)
    Bs = (ctypes.c_int * 2)(8, 12)
    Ms = (ctypes.c_int64 * 2)(10, 20)
    assert lib.sgl_batch_create(ctypes.byref(h), 0, Bs, Ms, 0, 0, 8, 2.0, 0, None) == 1
    assert h.value is None
    assert lib.sgl_batch_create(ctypes.byref(h), 2, None, Ms, 0, 0, 8, 2.0, 0, None) == 1
    bad = (ctypes.c_int * 2)(8, 0)
    assert lib.sgl_batch_create(ctypes.byref(h), 2, bad, Ms, 0, 0, 8, 2.0, 0, None) == 1
    assert "instance 1" in lib.sgl_last_error().decode()
    assert lib.sgl_batch_create(ctypes.byref(h), 2, Bs, Ms, 0, 0, 8, 2.0, 2, None) == 1     # profiling flag
    assert lib.sgl_batch_create(ctypes.byref(h), 2, Bs, Ms, 0, 0, 8, 2.0, 32, None) == 1    # overlapped binning
    assert "SGL_FLAG_OVERLAP_POINTS" in lib.sgl_last_error().decode()
    assert lib.sgl_batch_forward(None, None, None) == 1
    lib.sgl_batch_destroy(None)


def test_fault_injection_entry_points_without_cuda(lib):
    # the test hooks need a plan; the allocation injection is process-wide and one-shot
    assert lib.sgl_test_hooks(None, 0, 0) == 1
    assert lib.sgl_test_fail_alloc(0) == 0
    out = ctypes.c_void_p()
    assert lib.sgl_plan_create(ctypes.byref(out), 8, 10, 0, 0, 8, 2.0, 0, None) == 2      # SGL_ERR_ALLOC
    assert out.value is None
    assert lib.sgl_test_fail_alloc(-1) == 0
