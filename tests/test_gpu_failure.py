"""Failure paths on the GPU in the allowed forms (marked gpu): no fault, trap or hang is caused.

- A bounded device wait is made to run out: a test hook has the tensor-core kernels' prep warps
  withhold their operand arrival, with a short wait limit.  The kernel issues no tensor-core
  product, drains its loads, frees its tensor memory and returns; sgl_sync reports
  SGL_ERR_TIMEOUT, and the same plan (hooks cleared) and a fresh plan compute correctly again.
- A device allocation is made to fail (host-side injection): plan and batch creation return
  SGL_ERR_ALLOC at every allocation they make and leave the device's free memory as it was.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_1809_10786_gb300 as sgl
from paper_1809_10786_gb300 import binding, inputs
from oracle import direct

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)
TIMEOUT, ALLOC = 5, 2


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.mark.parametrize("call", ["forward", "grad_points"])
def test_withheld_arrival_times_out_and_the_plan_recovers(call):
    lib = binding.load_library()
    B, M = 16, 3001
    c = inputs.coefficients(B, 9600)
    x = inputs.points_gaussian(M, 9601)
    g = inputs.complex_normal(M, 9602)
    p = sgl.Plan(B, M, precision=sgl.PREC_FP32_MIXED, q=8, device=DEV)
    assert p.info()["tensor_cores"]["interp"] and p.info()["tensor_cores"]["grad"]
    p.set_points(gpu(x))
    run = (lambda: p.forward(gpu(c))) if call == "forward" else (lambda: p.grad_points(gpu(c), gpu(g)))
    assert lib.sgl_test_hooks(p._h, 1, 1 << 20) == 0          # about half a millisecond per wait
    run()
    with pytest.raises(sgl.SGLError) as ei:
        p.sync()
    assert ei.value.status == TIMEOUT
    # the same plan with the hooks cleared, and a fresh plan: correct again
    assert lib.sgl_test_hooks(p._h, 0, 0) == 0
    f_ref, _ = direct.forward(B, x, c)
    f = p.forward(gpu(c)).cpu().numpy()
    p.sync()
    assert rel(f, f_ref) <= 2e-6
    if call == "grad_points":
        g_ref, _ = direct.grad_points(B, x, c, g)
        gx = p.grad_points(gpu(c), gpu(g)).cpu().numpy()
        p.sync()
        ok = np.linalg.norm(x, axis=1) > 0.05 * p.rho()
        assert rel(gx[ok], g_ref[ok]) <= 1e-4
    q = sgl.Plan(B, M, precision=sgl.PREC_FP32_MIXED, q=8, device=DEV)
    q.set_points(gpu(x))
    assert rel(q.forward(gpu(c)).cpu().numpy(), f_ref) <= 2e-6
    q.sync()


def test_test_hooks_reject_unknown_bits():
    lib = binding.load_library()
    p = sgl.Plan(8, 10, device=DEV)
    assert lib.sgl_test_hooks(p._h, 2, 0) == 1
    assert lib.sgl_test_hooks(p._h, 0, -1) == 1


def _fail_every_allocation(create):
    """create() under an injected failure of its k-th device allocation, k = 0, 1, ... until it
    succeeds; returns the number of allocations it makes.  Every failure must be SGL_ERR_ALLOC."""
    lib = binding.load_library()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(DEV)
    try:
        for k in range(200):
            assert lib.sgl_test_fail_alloc(k) == 0
            try:
                obj = create()
            except sgl.SGLError as e:
                assert e.status == ALLOC, (k, e)
                continue
            lib.sgl_test_fail_alloc(-1)
            obj.close()
            torch.cuda.synchronize()
            assert torch.cuda.mem_get_info(DEV)[0] == free0        # nothing leaked by the failed attempts
            return k
        raise AssertionError("creation never succeeded")
    finally:
        lib.sgl_test_fail_alloc(-1)


def test_plan_creation_fails_cleanly_at_every_allocation():
    n = _fail_every_allocation(lambda: sgl.Plan(24, 5000, precision=sgl.PREC_FP32_MIXED, q=8, device=DEV, host_io=True))
    assert n >= 30                                                  # the plan's workspace buffers


def test_batch_creation_fails_cleanly_at_every_allocation():
    n = _fail_every_allocation(lambda: sgl.BatchPlan([8, 13, 5], [100, 300, 20], precision=sgl.PREC_FP64, q=6, device=DEV))
    assert n >= 60


def test_inverse_work_allocation_failure_is_reported():
    lib = binding.load_library()
    B, M = 5, 200
    x = inputs.points_gaussian(M, 9700)
    p = sgl.Plan(B, M, device=DEV)
    p.set_points(gpu(x))
    f = gpu(inputs.values(M, 9701))
    try:
        lib.sgl_test_fail_alloc(0)
        with pytest.raises(sgl.SGLError) as ei:
            p.inverse(f, iters=3)
        assert ei.value.status == ALLOC
    finally:
        lib.sgl_test_fail_alloc(-1)
    c, res, k = p.inverse(f, iters=3)                                 # works once allocation succeeds
    assert k == 3 and np.isfinite(res)
