#!/usr/bin/env python3
"""Benchmark of the NFSGLFT hot path on GB300: Mpoints/s at bandwidth B = 64.

One step = one pass of the whole path over M = 10^6 synthetic points:
  set_points (rho, transformed points, bin sort, radial matrices)
  + forward  (radial and polar conversions, pruned inverse FFT, interpolation)
  + adjoint  (spreading, pruned forward FFT, adjoint conversions; one all-reduce when N > 1)
  + point gradient (conversions, inverse FFT, window-derivative interpolation)
with sigma = 2, Kaiser-Bessel window, cutoff q = 8, run in the FP32-mixed precision
(the headline value) and in FP64 (reported beside it).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  Timing: CUDA events on the launching stream around
each step, an L2 flush (a 256 MiB write) between steps, outside the timed events.
"""
import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "NDSGLFT Mpoints/s at B=64 fwd/adj: FP32-mixed vs FP64 on GB300 at stated error"
UNIT = "Mpoints/s"
SM_COUNT = 152
FP32_LANES_PER_SM = 128          # FFMA lanes per SM
FP64_FMA_PER_SM_CLK = 2          # DFMA per SM per clock on GB300 (measured 1.0 TFLOP/s at ~1.9 GHz)
FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            return d, "measured"
        except Exception:
            pass
    return dict(FALLBACK), "fallback"


def alu_peaks(peaks):
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    fp32 = SM_COUNT * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
    fp64 = SM_COUNT * FP64_FMA_PER_SM_CLK * 2 * mhz * 1e6 / 1e12
    return fp32, fp64


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "50", "-i", str(gpu_index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(smax), "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- algorithmic work per stage
def stage_work(info, M, q, prec):
    """Algorithmic bytes (HBM-bound stages) or flops (ALU-bound stages) of one call of each stage."""
    B = info["B"]
    K0, K1 = 2 * B - 2, B - 1
    W = 2 * K1 + 1
    rows0, rows1, N2 = info["rows"][0], info["rows"][1], info["N"][2]
    cs = 8 if prec == "fp32_mixed" else 16
    taps = (2 * q) ** 3
    if info.get("sym_grid"):
        # symmetry-reduced passes: radial lines kappa1 >= 0 (K1 + 1), grid lines of
        # [0, N0/2] x [0, N1/2] (H0 x H1), the halo rows copied (forward) or folded (adjoint)
        H0, H1, K1p = info["N"][0] // 2 + 1, info["N"][1] // 2 + 1, K1 + 1
        halo = (rows0 * rows1 - H0 * H1) * N2 * cs
        fft_fwd = ((K0 + 1) * K1p * W * 16 + H0 * K1p * W * cs               # pass A: zeta in, X0 out
                   + H0 * K1p * W * cs + H0 * H1 * W * cs                    # pass B
                   + H0 * H1 * W * cs + H0 * H1 * N2 * cs                    # pass C
                   + 2 * halo)                                               # halo rows: read sources, write
        fft_adj = (3 * halo                                                  # halo fold: read, read + write partners
                   + H0 * H1 * N2 * cs + H0 * H1 * W * cs                    # pass C'
                   + H0 * H1 * W * cs + H0 * W * W * cs                      # pass B'
                   + H0 * W * W * cs + H0 * K1p * W * cs                     # kappa1 fold
                   + H0 * K1p * W * cs + (2 * K0 + 1) * K1p * W * 16)        # pass A'
    else:
        fft_fwd = ((K0 + 1) * (K1 + 1) * W * 16 + rows0 * W * W * cs          # pass A: zeta in, X0 out
                   + rows0 * W * W * cs + rows0 * rows1 * W * cs                # pass B
                   + rows0 * rows1 * W * cs + rows0 * rows1 * N2 * cs)          # pass C
        fft_adj = (rows0 * rows1 * N2 * cs + rows0 * rows1 * W * cs
                   + rows0 * rows1 * W * cs + rows0 * W * W * cs
                   + rows0 * W * W * cs + (2 * K0 + 1) * W * W * 16)
    radial = 4 * sum((K0 + 1) * (2 * l + 1) * (B - l) for l in range(B))
    polar = 4 * (K0 + 1) * (K1 + 1) * sum(B - abs(m) for m in range(-(B - 1), B))
    # FP64 plans run the three windowed loops in double-float arithmetic unless native: a
    # double-float multiply-add is 12 FP32-pipe instructions, so its ceiling is the FP32 peak / 12
    # in flops of the binary64 algorithm ("df")
    alu = {"fp32_mixed": "fp32", "fp64": "df", "fp64_native": "fp64"}[prec]
    # interpolation / gradient on the tensor cores (3xTF32 slab products): the algorithmic flops
    # stay the windowed sums' own; the peak is the TF32 one
    tc = info.get("tensor_cores", {})
    k_interp = "tf32" if tc.get("interp") else alu
    k_grad = "tf32" if tc.get("grad") else alu
    return {
        "points": ("hbm", M * (24 + 24 + 4)),
        "radial_matrix": ("fp64", 2 * (K0 + 1) * 2 * B * B * (B + 1) // 2),
        "radial": ("fp64", radial),
        "polar": ("fp64", polar),
        "fft_forward": ("hbm", fft_fwd),
        "interp": (k_interp, 4 * taps * M),
        "spread": (alu, 4 * taps * M),
        "fft_adjoint": ("hbm", fft_adj),
        "polar_adjoint": ("fp64", polar),
        "radial_adjoint": ("fp64", radial),
        "grad_interp": (k_grad, 12 * taps * M),
    }


def traffic_for(stage, prec):
    """DRAM bytes per launch of a stage from the committed ncu summary, if its kernel source is unchanged."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    try:
        rec = json.load(open(path)).get("%s/%s" % (prec, stage))
    except Exception:
        return None
    if not rec:
        return None
    src = os.path.join(ROOT, "paper_1809_10786_gb300", "csrc", rec["source"])
    if not os.path.exists(src) or hashlib.sha256(open(src, "rb").read()).hexdigest() != rec["source_sha256"]:
        return None
    return rec["bytes_per_launch_full_size"]


# ---------------------------------------------------------------- our arm
def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_1809_10786_gb300 as sgl
    from paper_1809_10786_gb300 import distributed as sd
    from paper_1809_10786_gb300 import inputs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world != args.gpus:
        raise SystemExit("--gpus %d but WORLD_SIZE %d" % (args.gpus, world))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    B, M, q = args.B, args.M, args.q
    c_h = inputs.coefficients(B, inputs.seed_for(2))
    x_h = inputs.points_gaussian(M, inputs.seed_for(2, 1 + rank))       # weak scaling: M points per rank
    y_h = inputs.values(M, inputs.seed_for(2, 100 + rank))
    g_h = inputs.complex_normal(M, inputs.seed_for(2, 200 + rank))
    c, x, y, g = (torch.from_numpy(a).to(dev) for a in (c_h, x_h, y_h, g_h))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    peaks, peak_src = load_peaks()
    fp32_peak, fp64_peak = alu_peaks(peaks)
    hbm_peak = float(peaks.get("hbm_gbs", FALLBACK["hbm_gbs"]))
    # dense TF32 = measured bf16 burst x the nominal TF32 / BF16 ratio (1.1 / 2.25 PFLOP/s)
    tf32_peak = float(peaks.get("bf16_tflops", FALLBACK["bf16_tflops"])) * (1.1 / 2.25)

    results = {}
    keep = {}
    precs = (("fp32_mixed", sgl.PREC_FP32_MIXED, False),) + (
        () if args.no_fp64 else (("fp64", sgl.PREC_FP64, False), ("fp64_native", sgl.PREC_FP64, True)))
    for prec_name, prec, native in precs:
        plan = sgl.Plan(B, M, precision=prec, window=sgl.WIN_KB, q=q, sigma=2.0, profile=True, device=dev,
                        native_fp64=native)
        out = {}

        def step():
            plan.set_points(x)
            out["f"], out["g"] = plan.forward_grad(c, g)      # forward values and point gradient, one pass
            a = plan.adjoint(y)
            out["a"] = sd.allreduce_coefficients(a)

        # clocks are sampled from the start of the warm-up (nvidia-smi needs a moment to start)
        # to the end of the timed steps
        sampler = ClockSampler(local) if prec_name == "fp32_mixed" else None
        for _ in range(args.warmup):
            step()
        barrier()
        plan.profile()                                    # drop warm-up stage times
        launches0 = plan.info()["kernel_launches"]
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        barrier()
        for k in range(args.steps):
            flush.zero_()                                  # evict L2 between steps (untimed)
            evs[k][0].record()
            step()
            evs[k][1].record()
        barrier()
        clocks = sampler.stop() if sampler else None
        ms = sum(a.elapsed_time(b) for a, b in evs)
        ms_max = sd.max_over_ranks(ms, dev)
        stages = plan.profile()
        launches = plan.info()["kernel_launches"] - launches0
        info = plan.info()
        work = stage_work(info, M, q, prec_name)
        table = {}
        for name, (t, n) in stages.items():
            if n == 0 or name not in work:
                continue
            kind, amount = work[name]
            per_launch_ms = t / n
            if kind == "hbm":
                achieved, peak, unit = amount / (per_launch_ms * 1e-3) / 1e9, hbm_peak, "GB/s"
            else:
                achieved = amount / (per_launch_ms * 1e-3) / 1e12
                peak, unit = {"fp32": fp32_peak, "fp64": fp64_peak, "tf32": tf32_peak, "df": fp32_peak / 12}[kind], "TFLOP/s"
            bound = "hbm" if kind == "hbm" else ("tensor" if kind == "tf32" else "alu")
            table[name] = {"ms": round(per_launch_ms, 4), "share": None, "bound": bound,
                           "alu": None if kind == "hbm" else kind, "achieved": round(achieved, 3), "peak": round(peak, 2),
                           "unit": unit, "frac": round(achieved / peak, 4), "algorithmic": amount}
        total_stage = sum(v["ms"] for v in table.values())
        for v in table.values():
            v["share"] = round(v["ms"] / total_stage, 4) if total_stage > 0 else None
        results[prec_name] = {"ms_per_step": ms_max / args.steps,
                              "value": world * M / (ms_max / args.steps * 1e-3) / 1e6,
                              "gpu_launches": launches, "stages": table, "clocks": clocks}
        keep[prec_name] = {k: v.detach().cpu().numpy() for k, v in out.items()}
        plan.close()
        del plan
        torch.cuda.empty_cache()

    # ---- the FP32-mixed path at the workload's other window cutoffs (same step, value only)
    by_q = {}
    if not args.no_extra_q:
        for qq in (4, 6):
            plan = sgl.Plan(B, M, precision=sgl.PREC_FP32_MIXED, window=sgl.WIN_KB, q=qq, sigma=2.0, device=dev)

            qout = {}

            def qstep():
                plan.set_points(x)
                qout["f"], _ = plan.forward_grad(c, g)
                sd.allreduce_coefficients(plan.adjoint(y))

            for _ in range(args.warmup):
                qstep()
            barrier()
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
            for k in range(args.steps):
                flush.zero_()
                evs[k][0].record()
                qstep()
                evs[k][1].record()
            barrier()
            ms = sd.max_over_ranks(sum(a.elapsed_time(b) for a, b in evs), dev)
            by_q[qq] = {"value": round(world * M / (ms / args.steps * 1e-3) / 1e6, 4), "ms_per_step": round(ms / args.steps, 4)}
            keep["fp32_mixed_q%d" % qq] = {"f": qout["f"].detach().cpu().numpy()}
            plan.close()
            del plan
            torch.cuda.empty_cache()

    # ---- per call, as the transform alone is usually timed: set_points + forward, and the adjoint
    # (same points), FP32-mixed and FP64 (value only)
    by_call = {}
    if not args.no_extra_q:
        for prec_name, prec in (("fp32_mixed", sgl.PREC_FP32_MIXED), ("fp64", sgl.PREC_FP64)):
            if prec_name == "fp64" and args.no_fp64:
                continue
            plan = sgl.Plan(B, M, precision=prec, window=sgl.WIN_KB, q=q, sigma=2.0, device=dev)
            plan.set_points(x)
            calls = {"set_points+forward": lambda: (plan.set_points(x), plan.forward(c)),
                     "adjoint": lambda: sd.allreduce_coefficients(plan.adjoint(y))}
            by_call[prec_name] = {}
            for name, fn in calls.items():
                for _ in range(args.warmup):
                    fn()
                barrier()
                evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
                for k in range(args.steps):
                    flush.zero_()
                    evs[k][0].record()
                    fn()
                    evs[k][1].record()
                barrier()
                ms = sd.max_over_ranks(sum(a.elapsed_time(b) for a, b in evs), dev)
                by_call[prec_name][name] = {"value": round(world * M / (ms / args.steps * 1e-3) / 1e6, 4),
                                            "ms": round(ms / args.steps, 4)}
            plan.close()
            del plan
            torch.cuda.empty_cache()

    # ---- inverse transform (iNFSGLFT) in the setup of the paper's last test (Sect. 8): Cartesian
    # grid G_N, N = 50 (M = 125000), kappa = 5, B = 8 and B = 16, CGNR from the mid-point rule, FP64;
    # errors as the paper measures them: max |c - c_true| and max |c - c_true| / |c_true|
    inverse_line = None
    if not args.no_inverse and rank == 0:
        Ni, kap = 50, 5.0
        tt = kap * (2.0 * np.arange(Ni) / Ni - 1.0)
        X, Y, Z = np.meshgrid(tt, tt, tt, indexing="ij")
        xg = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
        Mi = xg.shape[0]
        wts = torch.from_numpy((2.0 * kap / Ni) ** 3 * np.exp(-np.sum(xg * xg, axis=1))).to(dev)
        inverse_line = {"setup": "Sect. 8 last test: Cartesian grid G_N, N=50 (M=125000), kappa=5, KB q=8, sigma=2, FP64; "
                                 "CGNR (sgl_inverse) from the mid-point rule (sgl_midpoint_guess); samples from the FP64 "
                                 "forward transform of seeded random coefficients U[-1/2,1/2]^2"}
        # B = 8: a fixed budget of 200 iterations; B = 16: until the relative residual is 1e-4
        # (at most 600 iterations), reporting the iterations that took
        for Bi, iters, tol in ((8, 200, 0.0), (16, 600, 1e-4)):
            ip = sgl.Plan(Bi, Mi, precision=sgl.PREC_FP64, window=sgl.WIN_KB, q=8, sigma=2.0, device=dev)
            ip.set_points(torch.from_numpy(xg).to(dev))
            c_true = torch.from_numpy(inputs.coefficients(Bi, inputs.seed_for(5))).to(dev)
            f_in = ip.forward(c_true)
            c0 = ip.midpoint_guess(f_in, wts)
            ip.inverse(f_in, coef0=c0, iters=2)          # warm-up (work vectors)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ci, resi, ki = ip.inverse(f_in, coef0=c0, iters=iters, tol=tol, method="cgnr")
            torch.cuda.synchronize()
            el = time.perf_counter() - t0

            def errs(c):
                d = (c - c_true).abs()
                return [float(d.max()), float((d / c_true.abs()).max())]
            inverse_line["B=%d" % Bi] = {
                "Nc": int(ip.Nc), "iterations": ki, "iteration_budget": iters, "residual_target": tol,
                "ms_per_iteration": round(el / max(ki, 1) * 1e3, 3),
                "relative_residual": resi, "max_abs_rel_error_initial": errs(c0), "max_abs_rel_error_final": errs(ci)}
            ip.close()
            del ip
            torch.cuda.empty_cache()

    # ---- the batch workload (256 instances, B uniform in 8..48, M = 10^U[3,5], q = 8): forward +
    # adjoint of every instance on fixed points, graph-captured with the autotuned lane count
    # against one launch after another on a single lane; Mpoints/s = all instances' points / time
    batch_line = None
    if not args.no_batch and rank == 0:
        specs = inputs.batch_instances(256, inputs.seed_for(3))
        tot = sum(M for _, M in specs)
        bcs = [torch.from_numpy(inputs.coefficients(Bi, inputs.seed_for(3, 10 + i))).to(dev) for i, (Bi, _) in enumerate(specs)]
        bxs = [torch.from_numpy(inputs.points_gaussian(Mi, inputs.seed_for(3, 1000 + i))).to(dev) for i, (_, Mi) in enumerate(specs)]
        bys = [torch.from_numpy(inputs.values(Mi, inputs.seed_for(3, 2000 + i))).to(dev) for i, (_, Mi) in enumerate(specs)]
        bfo = [torch.empty(Mi, dtype=torch.complex128, device=dev) for _, Mi in specs]
        bao = [torch.empty(sgl.num_coeffs(Bi), dtype=torch.complex128, device=dev) for Bi, _ in specs]
        batch_line = {"workload": "256 instances, B uniform in 8..48, M = round(10^U[3,5]) (%d points in all), KB q=8, "
                                  "sigma=2; step = batch forward + batch adjoint on fixed points" % tot,
                      "unit": UNIT}
        for prec_name, prec in (("fp32_mixed", sgl.PREC_FP32_MIXED), ("fp64", sgl.PREC_FP64)):
            if prec_name == "fp64" and args.no_fp64:
                continue
            bp = sgl.BatchPlan([Bi for Bi, _ in specs], [Mi for _, Mi in specs], precision=prec, q=8, device=dev)
            bp.set_points(bxs)
            res = {}
            for mode in ("one_launch_per_instance", "graph_autotuned_lanes"):
                if mode == "graph_autotuned_lanes":
                    bp.use_graph(True)
                    lanes, _ = bp.autotune(None)
                else:
                    bp.use_graph(False)
                    bp.set_lanes(1)
                    lanes = 1
                for _ in range(args.warmup):
                    bp.forward(bcs, bfo)
                    bp.adjoint(bys, bao)
                barrier()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(args.steps):
                    bp.forward(bcs, bfo)
                    bp.adjoint(bys, bao)
                e1.record()
                barrier()
                ms = e0.elapsed_time(e1) / args.steps
                res[mode] = {"value": round(tot / (ms * 1e-3) / 1e6, 4), "ms_per_step": round(ms, 3), "lanes": lanes}
            batch_line[prec_name] = res
            bp.close()
            del bp
            torch.cuda.empty_cache()

    # ---- end to end through the C-ABI with host buffers (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        hplan = sgl.Plan(B, M, precision=sgl.PREC_FP32_MIXED, window=sgl.WIN_KB, q=q, sigma=2.0, host_io=True, device=dev)
        xp = torch.from_numpy(x_h).pin_memory()
        cp = torch.from_numpy(c_h).pin_memory()
        yp = torch.from_numpy(y_h).pin_memory()
        gp = torch.from_numpy(g_h).pin_memory()
        fo = torch.empty(M, dtype=torch.complex128).pin_memory()
        ao = torch.empty(hplan.Nc, dtype=torch.complex128).pin_memory()
        go = torch.empty((M, 3), dtype=torch.float64).pin_memory()

        def hstep():
            hplan.forward_grad_host(xp, cp, gp, fo, go)
            hplan.adjoint_host(None, yp, ao)            # same points: no second copy or binning

        for _ in range(args.warmup):
            hstep()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            hstep()
        barrier()
        el = sd.max_over_ranks(time.perf_counter() - t0, dev)
        Nc = hplan.Nc
        e2e = {"value": world * M / (el / args.steps) / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": 24 * M + 16 * Nc + 16 * M + 16 * M,
               "d2h_bytes_per_step": 16 * M + 24 * M + 16 * Nc,
               "path": "sgl_forward_grad_host (points, coefficients, gradient seeds in; values and point "
                       "gradient out) + sgl_adjoint_host on the same points (values in, coefficients out), "
                       "pinned host buffers"}
        hplan.close()

    head = results["fp32_mixed"]
    dom_name = max(head["stages"], key=lambda k: head["stages"][k]["ms"])
    dom = head["stages"][dom_name]
    traffic = traffic_for(dom_name, "fp32_mixed")
    roofline = {"kernel": dom_name, "bound": dom["bound"], "achieved": dom["achieved"], "peak": dom["peak"],
                "unit": dom["unit"], "frac": dom["frac"], "traffic": traffic,
                "peak_source": (peak_src if dom["bound"] == "hbm" else
                                "measured bf16 burst x 1.1/2.25 (nominal TF32 : BF16)" if dom["bound"] == "tensor" else
                                "derived: 152 SMs x %s x 2 flop x %.0f MHz" % (
                                    "128 FFMA lanes" if dom["alu"] == "fp32" else "2 DFMA", float(peaks.get("sm_max_mhz", 2070))))}

    line = {"metric": METRIC, "value": round(head["value"], 4), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(head["ms_per_step"], 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "fp32_mixed_vs_fp64": None if "fp64" not in results else {
                "fp64_double_float_loops": {"value": round(results["fp64"]["value"], 4),
                                            "ratio": round(head["value"] / results["fp64"]["value"], 3)},
                "fp64_binary64_loops": {"value": round(results["fp64_native"]["value"], 4),
                                        "ratio": round(head["value"] / results["fp64_native"]["value"], 3)},
                "note": "same step; FP64 plan = binary64 everywhere except the three windowed loops, which run in "
                        "double-float (default) or binary64 (SGL_FLAG_NATIVE_FP64) arithmetic"},
            "data": "synthetic (seeded): coefficients U[-1/2,1/2]^2, points N(0, I/2) in |x| <= 5, values U[-1/2,1/2]^2",
            "config": {"workload": "B=64 (Nc=89440), M=1e6 points per GPU, sigma=2, Kaiser-Bessel q=8; step = set_points"
                                   " + forward values with point gradient (sgl_forward_grad, one pass) + adjoint",
                       "B": B, "M_per_gpu": M, "q": q, "sigma": 2.0, "window": "kaiser-bessel",
                       "precision": "fp32-mixed (FFT, spreading, interpolation in FP32; conversions FP64)",
                       "parallelism": "points sharded, adjoint coefficients all-reduced" if world > 1 else "single GPU",
                       "l2": "256 MiB write between timed steps (flush), inputs and grid exceed L2 in total"},
            "gpu_launches": head["gpu_launches"],
            "roofline": roofline, "clocks": head["clocks"],
            "fp64": None if "fp64" not in results else {
                "value": round(results["fp64"]["value"], 4), "unit": UNIT, "ms_per_step": round(results["fp64"]["ms_per_step"], 4),
                "precision": "FP64 plan (binary64 everywhere but the windowed loops, which run in double-float "
                             "arithmetic: FP32 pairs with error-free products and sums)",
                "gpu_launches": results["fp64"]["gpu_launches"], "stages": results["fp64"]["stages"]},
            "fp64_native": None if "fp64_native" not in results else {
                "value": round(results["fp64_native"]["value"], 4), "unit": UNIT,
                "ms_per_step": round(results["fp64_native"]["ms_per_step"], 4),
                "precision": "FP64 plan with SGL_FLAG_NATIVE_FP64 (binary64 windowed loops)",
                "gpu_launches": results["fp64_native"]["gpu_launches"],
                "stages": {k: v["ms"] for k, v in results["fp64_native"]["stages"].items()}},
            "stages_fp32_mixed": head["stages"],
            "fp32_mixed_other_cutoffs": by_q,
            "by_call": by_call,
            "inverse": inverse_line,
            "batch": batch_line,
            "e2e": e2e}

    # ---- CPU baseline (oracle on the host cores, rank 0, N = 1) and the measured error on its sample
    if rank == 0 and world == 1 and not args.no_cpu:
        base, err = cpu_baseline(args, x_h, c_h, y_h, g_h, keep, dev)
        for qq in by_q:
            if ("fp32_mixed_q%d" % qq) in err:
                by_q[qq]["forward_error"] = err["fp32_mixed_q%d" % qq]["forward"]
        line["cpu_baseline"] = base
        line["error_vs_oracle"] = err
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def cpu_baseline(args, x_h, c_h, y_h, g_h, keep, dev):
    """Oracle (direct sum) timed on a bounded sample; its outputs also give the GPU error on that sample."""
    import numpy as np
    import torch

    import paper_1809_10786_gb300 as sgl
    from oracle import direct

    S = args.cpu_sample
    idx = np.arange(S)
    xs = np.ascontiguousarray(x_h[idx])
    t0 = time.perf_counter()
    f_ref, threads = direct.forward(args.B, xs, c_h)
    a_ref, _ = direct.adjoint(args.B, xs, y_h[idx])
    g_ref, _ = direct.grad_points(args.B, xs, c_h, g_h[idx])
    el = time.perf_counter() - t0
    base = {"value": round(S / el / 1e6, 8), "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "%d of the %d points (forward + adjoint + point gradient, direct sum, FP64); %.1f s" % (S, args.M, el)}
    err = {}
    for prec_name, prec, native in (("fp32_mixed", sgl.PREC_FP32_MIXED, False), ("fp64", sgl.PREC_FP64, False),
                                    ("fp64_native", sgl.PREC_FP64, True)):
        if prec_name not in keep:
            continue
        k = keep[prec_name]
        ef = np.abs(k["f"][idx] - f_ref).max() / np.abs(f_ref).max()
        eg = np.abs(k["g"][idx] - g_ref).max() / np.abs(g_ref).max()
        # adjoint on the sample alone: same plan type, values zero outside the sample
        plan = sgl.Plan(args.B, args.M, precision=prec, window=sgl.WIN_KB, q=args.q, sigma=2.0, device=dev,
                        native_fp64=native)
        plan.set_points(torch.from_numpy(x_h).to(dev))
        ym = np.zeros_like(y_h)
        ym[idx] = y_h[idx]
        a = plan.adjoint(torch.from_numpy(ym).to(dev)).cpu().numpy()
        plan.close()
        ea = np.abs(a - a_ref).max() / np.abs(a_ref).max()
        err[prec_name] = {"forward": float(ef), "adjoint": float(ea), "grad": float(eg),
                          "measure": "max |gpu - oracle| / max |oracle| on the sample"}
    for key in sorted(k for k in keep if k.startswith("fp32_mixed_q")):
        ef = np.abs(keep[key]["f"][idx] - f_ref).max() / np.abs(f_ref).max()
        err[key] = {"forward": float(ef), "measure": "max |gpu - oracle| / max |oracle| on the sample"}
    return base, err


# ---------------------------------------------------------------- reference arm (the oracle)
def run_reference(args):
    import numpy as np

    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import direct
    from paper_1809_10786_gb300 import inputs

    S = args.ref_sample
    B = args.B
    c = inputs.coefficients(B, inputs.seed_for(2))
    x = inputs.points_gaussian(S, inputs.seed_for(2, 1))
    y = inputs.values(S, inputs.seed_for(2, 100))
    g = inputs.complex_normal(S, inputs.seed_for(2, 200))

    def step():
        _, t = direct.forward(B, x, c)
        direct.adjoint(B, x, y)
        direct.grad_points(B, x, c, g)
        return t

    for _ in range(args.warmup):
        threads = step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        threads = step()
    el = (time.perf_counter() - t0) / args.steps
    value = S / el / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 8), "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(el * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded), same generators",
            "config": {"workload": "B=64 (Nc=89440), sample of %d of the 1e6 points per step; step = forward + adjoint"
                                   " + point gradient by direct summation (the CPU oracle)" % S,
                       "B": B, "M_sample": S},
            "cpu_baseline": {"value": round(value, 8), "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": "%d points per step" % S},
            "e2e": {"value": round(value, 8), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--B", type=int, default=64)
    ap.add_argument("--M", type=int, default=1_000_000)
    ap.add_argument("--q", type=int, default=8)
    ap.add_argument("--cpu-sample", type=int, default=96000)
    ap.add_argument("--ref-sample", type=int, default=24000)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extra-q", action="store_true")
    ap.add_argument("--no-inverse", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 256-instance batch leg")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison run (profiling captures)")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
