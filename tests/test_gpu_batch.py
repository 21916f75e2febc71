"""Batched transforms (marked gpu): a batch gives the same results as one plan per
instance, with and without CUDA-graph replay, for any number of concurrent lanes; the
256-instance workload (B uniform in 8..48, M log-uniform in [1e3, 1e5]) matches the oracle on
sampled outputs of 64 instances, forward and adjoint; the autotuner's choice is cached."""
import json
import os

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


def instances(specs, seed):
    cs = [inputs.coefficients(B, seed + 10 * i) for i, (B, M) in enumerate(specs)]
    xs = [inputs.points_gaussian(M, seed + 10 * i + 1) for i, (B, M) in enumerate(specs)]
    ys = [inputs.values(M, seed + 10 * i + 2) for i, (B, M) in enumerate(specs)]
    return cs, xs, ys


@pytest.mark.parametrize("lanes", [1, 3, 6])
@pytest.mark.parametrize("prec", [sgl.PREC_FP64, sgl.PREC_FP32_MIXED])
def test_batch_matches_single_plans_and_graph_replay(prec, lanes):
    specs = [(8, 900), (13, 1500), (21, 40), (37, 3000), (8, 1), (16, 700)]
    cs, xs, ys = instances(specs, 8100)
    bp = sgl.BatchPlan([B for B, _ in specs], [M for _, M in specs], precision=prec, q=6)
    assert bp.lanes() == 6                                    # min(n, 8) to start with
    bp.set_lanes(lanes)
    assert bp.lanes() == lanes
    bp.set_points([gpu(x) for x in xs])
    f_b = [t.cpu().numpy() for t in bp.forward([gpu(c) for c in cs])]
    a_b = [t.cpu().numpy() for t in bp.adjoint([gpu(y) for y in ys])]
    for i, (B, M) in enumerate(specs):
        p = sgl.Plan(B, M, precision=prec, q=6)
        p.set_points(gpu(xs[i]))
        f = p.forward(gpu(cs[i])).cpu().numpy()
        a = p.adjoint(gpu(ys[i])).cpu().numpy()
        assert np.array_equal(f_b[i], f)
        # spreading adds with atomics: the order (and FP32 rounding) differs from run to run
        tol = 1e-12 if prec == sgl.PREC_FP64 else 2e-7          # FP32: measured at most 3.3e-8
        check("batch adjoint vs plan prec=%d i=%d" % (prec, i), np.abs(a_b[i] - a).max() / max(np.abs(a).max(), 1e-300), tol)
    # graph mode: capture once, replay, same numbers; new pointers recapture
    bp.use_graph(True)
    ct = [gpu(c) for c in cs]
    outs = [torch.empty(M, dtype=torch.complex128, device=DEV) for _, M in specs]
    for _ in range(3):
        bp.forward(ct, outs)
    torch.cuda.synchronize()
    for i in range(len(specs)):
        assert np.array_equal(outs[i].cpu().numpy(), f_b[i])
    assert bp.info()["graph_launches"] == 3
    f_new = [t.cpu().numpy() for t in bp.forward(ct)]
    for i in range(len(specs)):
        assert np.array_equal(f_new[i], f_b[i])
    bp.sync()


# FP32: forward measured <= 1.2e-6 on 12 instances
@pytest.mark.parametrize("prec,tol_f,tol_a", [(sgl.PREC_FP64, 1e-10, 1e-10), (sgl.PREC_FP32_MIXED, 6e-6, 1e-6)])
def test_256_instance_workload_sampled(prec, tol_f, tol_a):
    specs = inputs.batch_instances(256, inputs.seed_for(3))
    cs, xs, ys = instances(specs, inputs.seed_for(3, 1))
    bp = sgl.BatchPlan([B for B, _ in specs], [M for _, M in specs], precision=prec, q=8)
    bp.set_points([gpu(x) for x in xs])
    bp.use_graph(True)
    rng = np.random.default_rng(3)
    picked = rng.choice(256, 64, replace=False)
    samples = {i: np.sort(rng.choice(specs[i][1], min(specs[i][1], 40), replace=False)) for i in picked}
    fs = [t.cpu().numpy() for t in bp.forward([gpu(c) for c in cs])]
    # adjoint of values that are zero outside each instance's sample (the oracle sums those only)
    ym = []
    for i, (B, M) in enumerate(specs):
        y = np.zeros(M, dtype=np.complex128)
        if i in samples:
            y[samples[i]] = ys[i][samples[i]]
        ym.append(y)
    as_ = [t.cpu().numpy() for t in bp.adjoint([gpu(y) for y in ym])]
    bp.sync()
    for i in picked:
        B, M = specs[i]
        idx = samples[i]
        ref, _ = direct.forward(B, xs[i][idx], cs[i])
        check("batch 256 forward prec=%d i=%d" % (prec, i), np.abs(fs[i][idx] - ref).max() / np.abs(ref).max(), tol_f)
        aref, _ = direct.adjoint(B, xs[i][idx], ys[i][idx])
        check("batch 256 adjoint prec=%d i=%d" % (prec, i), np.abs(as_[i] - aref).max() / np.abs(aref).max(), tol_a)


def test_autotune_chooses_lanes_and_caches_them(tmp_path):
    specs = inputs.batch_instances(24, inputs.seed_for(3, 7))
    cs, xs, ys = instances(specs, 8300)
    cache = str(tmp_path / "lanes.json")
    bp = sgl.BatchPlan([B for B, _ in specs], [M for _, M in specs], precision=sgl.PREC_FP32_MIXED, q=6)
    bp.set_points([gpu(x) for x in xs])
    bp.use_graph(True)
    L, ms = bp.autotune(cache)
    assert 1 <= L <= 24 and ms > 0 and bp.lanes() == L
    entry = list(json.load(open(cache)).values())
    assert len(entry) == 1 and entry[0]["lanes"] == L and set(entry[0]["ms"]) == {"1", "2", "4", "8", "16"}
    f = [t.cpu().numpy() for t in bp.forward([gpu(c) for c in cs])]
    # a second batch of the same instances takes the cached choice without timing
    bp2 = sgl.BatchPlan([B for B, _ in specs], [M for _, M in specs], precision=sgl.PREC_FP32_MIXED, q=6)
    L2, ms2 = bp2.autotune(cache)
    assert L2 == L and ms2 == -1.0 and bp2.lanes() == L
    bp2.set_points([gpu(x) for x in xs])
    f2 = [t.cpu().numpy() for t in bp2.forward([gpu(c) for c in cs])]
    for a, b in zip(f, f2):
        assert np.array_equal(a, b)
    bp.sync()
    bp2.sync()


def test_set_lanes_rejects_bad_counts():
    bp = sgl.BatchPlan([8, 9, 10], [10, 10, 10], device=DEV)
    for bad in (0, 4, 33):
        with pytest.raises(sgl.SGLError) as ei:
            bp.set_lanes(bad)
        assert ei.value.status == 1
