"""The allocation-free entry point, sgl_trig_coeffs_noalloc (marked gpu).

Callers that own all of their device memory through their own allocator, or run
under a fixed device-memory budget, cannot let a library call cudaMalloc; this entry
point serves them with static scratch.  It must give the same trigonometric
coefficients as the plan-based sgl_trig_coeffs, call after call (the scratch array
is shared and keeps the previous call's contents), and reject sizes beyond its
static limit.  This file is collected last so a failure here leaves every other
test already run.
"""
import numpy as np
import pytest
import torch

import paper_1809_10786_gb300 as sgl
from paper_1809_10786_gb300 import binding, inputs

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


def _reference(B, x, c):
    p = sgl.Plan(B, x.shape[0], q=min(8, B))
    p.set_points(x)
    eta = p.trig_coeffs(c)
    torch.cuda.synchronize()
    return eta.cpu().numpy()


@pytest.mark.parametrize("B,M", [(8, 1000), (binding.NOALLOC_MAX_B, 5000), (3, 17)])
def test_matches_plan_entry_point_on_two_calls_in_a_row(B, M):
    results = []
    for call in range(2):
        c = torch.from_numpy(inputs.coefficients(B, 900 + 10 * B + call)).to(DEV)
        x = torch.from_numpy(inputs.points_gaussian(M, 901 + 10 * B + call)).to(DEV)
        got = binding.trig_coeffs_noalloc(B, x, c)
        torch.cuda.synchronize()
        ref = _reference(B, x, c)
        err = np.abs(got.cpu().numpy() - ref).max() / np.abs(ref).max()
        assert err <= 1e-13, (call, err)
        results.append(got.cpu().numpy())
    assert not np.array_equal(results[0], results[1])      # two different problems, both right


def test_rejects_bandwidth_above_static_limit():
    B = binding.NOALLOC_MAX_B + 1
    c = torch.zeros(sgl.num_coeffs(B), dtype=torch.complex128, device=DEV)
    x = torch.zeros((4, 3), dtype=torch.float64, device=DEV)
    with pytest.raises(sgl.SGLError) as ei:
        binding.trig_coeffs_noalloc(B, x, c)
    assert ei.value.status == 1
    assert str(binding.NOALLOC_MAX_B) in str(ei.value)
