"""The allocation-free entry point, sgl_trig_coeffs_noalloc (marked gpu).

Callers that own all of their device memory through their own allocator, or run
under a fixed device-memory budget, cannot let a library call cudaMalloc; this entry
point serves them with static scratch.  It must give the trigonometric coefficients
of the exact factorization (the oracle's, and the plan-based sgl_trig_coeffs's),
call after call (the scratch array is shared and keeps the previous call's contents),
allocate nothing on the device, and reject sizes beyond its static limit.  This file
is collected last so a failure here leaves every other test already run.
"""
import numpy as np
import pytest
import torch

import paper_1809_10786_gb300 as sgl
from paper_1809_10786_gb300 import binding, inputs
from oracle import factorization as fz

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)
MAXB = binding.noalloc_max_b()


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def _plan_eta(B, x, c):
    p = sgl.Plan(B, max(x.shape[0], 1), q=min(8, B))
    p.set_points(x)
    eta = p.trig_coeffs(c).cpu().numpy()
    rho = p.rho()
    p.close()
    return eta, rho


def _oracle_eta(B, c, rho):
    # the oracle's eta on |k0| <= 2B-2, |k1|, |k2| <= B-1 (the exported support)
    ref = fz.eta(B, c, rho)
    K0, K1 = 2 * B - 2, B - 1
    return ref[2 * B - K0:2 * B + K0 + 1, 2 * B - K1:2 * B + K1 + 1, 2 * B - K1:2 * B + K1 + 1]


@pytest.mark.parametrize("B,M", [(8, 1000), (MAXB, 5000), (3, 17), (5, 0)])
def test_matches_oracle_and_plan_on_two_calls_in_a_row(B, M):
    results = []
    for call in range(2):
        c_h = inputs.coefficients(B, 900 + 10 * B + call)
        c = torch.from_numpy(c_h).to(DEV)
        x = torch.from_numpy(inputs.points_gaussian(M, 901 + 10 * B + call)).to(DEV).reshape(M, 3)
        got = binding.trig_coeffs_noalloc(B, x, c).cpu().numpy()
        ref, rho = _plan_eta(B, x, c)
        assert rel(got, ref) <= 1e-13, (call, rel(got, ref))
        assert rel(got, _oracle_eta(B, c_h, rho)) <= 1e-12
        results.append(got)
    assert not np.array_equal(results[0], results[1])      # two different problems, both right


def test_second_call_allocates_no_device_memory():
    # after the first call (set-up), a call with the output passed in changes neither the
    # device's free memory nor torch's allocator
    B, M = 16, 4000
    c = torch.from_numpy(inputs.coefficients(B, 77)).to(DEV)
    x = torch.from_numpy(inputs.points_gaussian(M, 78)).to(DEV)
    out = torch.empty((4 * B - 3, 2 * B - 1, 2 * B - 1), dtype=torch.complex128, device=DEV)
    binding.trig_coeffs_noalloc(B, x, c, out=out)
    torch.cuda.synchronize()
    first = out.clone()
    free0, _ = torch.cuda.mem_get_info(DEV)
    alloc0, reserved0 = torch.cuda.memory_allocated(DEV), torch.cuda.memory_reserved(DEV)
    binding.trig_coeffs_noalloc(B, x, c, out=out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(DEV)
    assert free1 == free0
    assert torch.cuda.memory_allocated(DEV) == alloc0 and torch.cuda.memory_reserved(DEV) == reserved0
    assert torch.equal(out, first)                      # same inputs, same result from the reused scratch


def test_rejects_bandwidth_above_static_limit():
    assert MAXB == 32                                   # the limit include/sgl.h states
    B = MAXB + 1
    c = torch.zeros(sgl.num_coeffs(B), dtype=torch.complex128, device=DEV)
    x = torch.zeros((4, 3), dtype=torch.float64, device=DEV)
    with pytest.raises(sgl.SGLError) as ei:
        binding.trig_coeffs_noalloc(B, x, c)
    assert ei.value.status == 1
    assert str(MAXB) in str(ei.value)
