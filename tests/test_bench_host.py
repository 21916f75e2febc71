"""Host logic of bench.py (CPU only): the algorithmic work behind each roofline fraction against
closed forms, the DRAM-traffic lookup keyed by the kernel source's hash, the clock sampler's
parsing of nvidia-smi output, and the derived ALU peaks."""
import hashlib
import json
import os

import pytest

import bench


def plan_info(B, q, sym_grid):
    # a B, sigma = 2 plan's report: n = (4B, 2B, 2B) oversampled twice, axes 0 and 1 windowed
    # (N/2 + 2q + 1 stored rows), axis 2 periodic
    N = [8 * B, 4 * B, 4 * B]
    return {"B": B, "N": N, "rows": [N[0] // 2 + 2 * q + 1, N[1] // 2 + 2 * q + 1, N[2]],
            "sym_grid": sym_grid, "tensor_cores": {"interp": True, "grad": True}}


def num_coeffs(B):
    return B * (B + 1) * (2 * B + 1) // 6


@pytest.mark.parametrize("B", [8, 21, 64])
def test_conversion_flops_match_closed_forms(B):
    w = bench.stage_work(plan_info(B, 8, True), 1000, 8, "fp32_mixed")
    # polar: kappa0 in [-(2B-2), 2B-2] x kappa1 in [0, B-1] x sum over m of the B - |m| degrees
    # l >= |m| is B^2, 4 flops per real-times-complex multiply-add
    assert w["polar"] == ("fp64", 4 * (2 * B - 1) * B * B * B)
    assert w["polar_adjoint"] == w["polar"]
    # radial: sum_l (2l + 1)(B - l) = B (B + 1)(2B + 1) / 6, the number of coefficients
    assert w["radial"] == ("fp64", 4 * (2 * B - 1) * num_coeffs(B))
    assert w["radial_adjoint"] == w["radial"]
    # radial matrices: 2B samples per entry, (2B - 1) kappa0 x (B - l) degrees for each l
    assert w["radial_matrix"] == ("fp64", 2 * (2 * B - 1) * 2 * B * (B * (B + 1) // 2))


@pytest.mark.parametrize("q,prec,alu", [(8, "fp32_mixed", "fp32"), (6, "fp64", "df"), (4, "fp64_native", "fp64")])
def test_windowed_loop_flops(q, prec, alu):
    M = 12345
    info = plan_info(32, q, True)
    info["tensor_cores"] = {}
    w = bench.stage_work(info, M, q, prec)
    taps = (2 * q) ** 3
    assert w["spread"] == (alu, 4 * taps * M)          # one complex-times-real multiply-add per tap
    assert w["interp"] == (alu, 4 * taps * M)
    assert w["grad_interp"] == (alu, 12 * taps * M)    # the value and two more derivative sums per tap
    assert w["points"] == ("hbm", 52 * M)              # xyz in, sorted coordinates and index out


def test_tensor_core_stages_take_the_tf32_peak():
    w = bench.stage_work(plan_info(64, 8, True), 10, 8, "fp32_mixed")
    assert w["interp"][0] == "tf32" and w["grad_interp"][0] == "tf32" and w["spread"][0] == "fp32"


@pytest.mark.parametrize("B", [16, 64])
def test_reduced_grid_fft_bytes(B):
    full = bench.stage_work(plan_info(B, 8, False), 1, 8, "fp32_mixed")
    half = bench.stage_work(plan_info(B, 8, True), 1, 8, "fp32_mixed")
    for stage in ("fft_forward", "fft_adjoint"):
        assert full[stage][0] == half[stage][0] == "hbm"
    # forward: the reduced passes store the lines of [0, N0/2] x [0, N1/2] (plus the mirrored
    # halo rows) instead of every stored line; pass C alone moves those lines in and out once
    assert half["fft_forward"][1] < full["fft_forward"][1]
    info = plan_info(B, 8, True)
    H0, H1 = info["N"][0] // 2 + 1, info["N"][1] // 2 + 1
    assert half["fft_forward"][1] > 2 * H0 * H1 * info["N"][2] * 8
    # adjoint: the two folds (halo rows, kappa1 < 0) are extra passes over the grid, so the
    # reduced adjoint moves about as many bytes as the full one although it transforms fewer lines
    assert 0.8 < half["fft_adjoint"][1] / full["fft_adjoint"][1] < 1.25


def test_traffic_lookup_follows_the_source_hash(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_1809_10786_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    src = csrc / "k.cu"
    src.write_bytes(b"__global__ void k() {}\n")
    rec = {"fp32_mixed/spread": {"kernel": "k", "source": "k.cu",
                                 "source_sha256": hashlib.sha256(src.read_bytes()).hexdigest(),
                                 "dram_read": 100, "dram_write": 20, "bytes_per_launch_full_size": 120}}
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_for("spread", "fp32_mixed") == 120
    assert bench.traffic_for("grad_interp", "fp32_mixed") is None        # no record
    src.write_bytes(b"__global__ void k() { /* changed */ }\n")
    assert bench.traffic_for("spread", "fp32_mixed") is None             # counters taken on other code
    os.remove(tmp_path / "profiles" / "ncu_traffic.json")
    assert bench.traffic_for("spread", "fp32_mixed") is None


class FakePopen:
    def __init__(self, out):
        self.out = out

    def terminate(self):
        pass

    def communicate(self, timeout=None):
        return self.out, ""


def sampler_with(monkeypatch, out):
    monkeypatch.setattr(bench.subprocess, "Popen", lambda *a, **k: FakePopen(out))
    return bench.ClockSampler(0)


def test_clock_sampler_reports_median_and_reasons(monkeypatch):
    na = "Not Active"
    lines = ["0, 2070, 2070, 900.1, 0x0, %s, %s, %s, %s" % (na, na, na, na),
             "0, 1980, 2070, 1390.0, 0x4, %s, %s, %s, Active" % (na, na, na),
             "0, 2055, 2070, 1200.0, 0x0, %s, %s, %s, %s" % (na, na, na, na),
             "garbage line"]
    r = sampler_with(monkeypatch, "\n".join(lines)).stop()
    assert r == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}


def test_clock_sampler_flags_thermal_slowdown_and_empty_output(monkeypatch):
    line = "0, 1500, 2070, 1400.0, 0x40, Not Active, Active, Not Active, Not Active"
    assert sampler_with(monkeypatch, line).stop()["reasons"] == ["hw_thermal_slowdown"]
    assert sampler_with(monkeypatch, "").stop()["reasons"] == ["no samples"]


def test_derived_alu_peaks():
    fp32, fp64 = bench.alu_peaks({"sm_max_mhz": 2070.0})
    assert fp32 == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12)      # 80.55 TFLOP/s
    assert fp64 == pytest.approx(152 * 2 * 2 * 2.07e9 / 1e12)        # 1.26 TFLOP/s
