#!/usr/bin/env python
"""Benchmark of the dust equilibrium-temperature + emission hot path on GB300.

One step = one dust_solve over the 2^18-cell, 200-wavelength, 96-grain
workload (absorbed powers -> temperatures -> SED -> energy-balance residual)
with inputs resident in device memory (J is 210 MB, larger than L2).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  `value` is whole-job grain-temperature solves per
second of the full path in the mixed-precision (BF16x3) form; the FP32 path,
the temperature-only rates, the SED cells/s and the errors against the FP64
oracle are reported beside it.  Under torchrun every rank solves its own
batch (weak scaling, no data-path collective).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "grain-T solves/s & SED cells/s, mixed vs FP32 at stated err, 1 GB300; p99 ms"
UNIT = "grain-T solves/s"
CONFIG_ID = 1
WORKLOAD = "2^18 cells x 200 wavelengths (0.09-1000 um) x 96 grains (3 species x 32 sizes), P_g(T) table 4096 pts"
# DRAM traffic (ncu dram__bytes_read.sum + dram__bytes_write.sum) of one launch,
# recorded from the capture in the named profile summary, with a hash of the
# kernel's sources at capture time: a run reports the figure only while the
# sources still hash the same, and null (with the reason) once they changed.
KERNEL_SOURCES = {
    "k_solve_emit": ["solve_emit.cu", "solve_core.cuh", "dust_internal.cuh", "mbar.cuh"],
    "k_emit": ["solve_emit.cu", "solve_core.cuh", "dust_internal.cuh", "mbar.cuh"],
    "k_fluct": ["fluct.cu", "solve_core.cuh", "dust_internal.cuh"],
}
RECORDED_TRAFFIC = {
    # kernel: (bytes per launch on the bench's workload, profile summary, sources sha256[:16])
    "k_solve_emit": (234.642176e6 + 358.232064e6, "profiles/k_solve_emit_2e18cells_K200_G96.md", "1b2b671c702a6864"),
    "k_emit": (220.631808e6 + 218.775808e6, "profiles/k_emit_2e18cells_K200_G96.md", "1b2b671c702a6864"),
    # the full-size launch, DRAM counters only (one ncu pass; the 2^14-cell --set full capture is in the same file)
    "k_fluct": (255.956992e6 + 175.320064e6, "profiles/k_fluct_2e14cells_K200_G36_M128.md", "2eac562135043b6a"),
}


def _measured_hbm_peak():
    """HBM copy bandwidth (GB/s) measured on this machine's GPUs, else the profiling fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            v = float(json.load(f)["hbm_gbs"])
        return v, "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError, TypeError):
        return 6800.0, "fallback 6.8 TB/s (no measured peak found)"


HBM_PEAK, HBM_PEAK_SOURCE = _measured_hbm_peak()


def _measured_bf16_peaks():
    """Dense BF16 tensor throughput (TF/s) measured on this machine's GPUs: burst and sustained."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["bf16_tflops"]), float(d["bf16_tflops_sustained"]), "measured (MEASURED_PEAKS.json)"
    except (OSError, KeyError, ValueError, TypeError):
        return 1900.0, 1700.0, "fallback 1.9 / 1.7 PF/s"


BF16_BURST, BF16_SUSTAINED, BF16_SOURCE = _measured_bf16_peaks()


def kernel_sources_sha(kernel):
    import hashlib

    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_0907_3768_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel):
    """(bytes or None, note) for the kernel's recorded ncu traffic."""
    nbytes, prof, sha = RECORDED_TRAFFIC[kernel]
    now = kernel_sources_sha(kernel)
    if nbytes is None or sha is None:
        return None, f"not captured for the current sources (sha {now})"
    if sha != now:
        return None, f"sources changed since the capture in {prof} (sha {sha}, now {now})"
    return nbytes, f"ncu capture in {prof} (sources sha {sha})"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", default="bf16x3")
    ap.add_argument("--paths", default="fp32,bf16x3,fp16x3", help="precisions to measure")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--cpu-interp-seconds", type=float, default=4.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer measurement")
    ap.add_argument("--no-serving", action="store_true", help="skip the request-stream measurement")
    ap.add_argument("--no-large", action="store_true", help="skip the 2^20-cell, K=500, G=240 solve")
    ap.add_argument("--no-ablation", action="store_true", help="skip the paper's kernel-3 Newton solve")
    ap.add_argument("--no-coupled", action="store_true", help="skip the self-absorbing (coupled) solve")
    ap.add_argument("--no-mass", action="store_true", help="skip the dust-mass form n[c,g] = n_g m_c")
    ap.add_argument("--no-fused", action="store_true", help="skip the fused absorption + solve kernel")
    ap.add_argument("--no-fluct", action="store_true", help="skip the thermally fluctuating grains")
    ap.add_argument("--no-sweep", action="store_true",
                    help="skip the time-per-call sweep over cell counts (also skipped by --no-e2e)")
    ap.add_argument("--fluct-levels", type=int, default=128)
    ap.add_argument("--profile-case", choices=["main", "main-two-kernel", "large", "fluct"], default=None,
                    help="no measurement: run --steps solves of one case for a profiler to capture "
                         "(main: 2^18 x 200 x 96 BF16x3, default kernels; main-two-kernel: the same with the solve "
                         "and the emission as two kernels; large: --large-cells x 500 x 240; fluct: "
                         "--profile-cells x 200 x 36 fluctuating grains on 128 levels)")
    ap.add_argument("--profile-cells", type=int, default=1 << 14)
    ap.add_argument("--large-cells", type=int, default=1 << 20,
                    help="cells of the K=500, G=240 solve (the full case is 2^20; fewer for profiling captures)")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-load", type=float, default=0.7, help="arrival rate / saturated throughput")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def shard_seed(rank):
    """Seed of rank `rank`'s batch: every rank solves its own full-size batch
    of independent cells (weak scaling), so no data crosses ranks."""
    import synth

    return synth.CONFIGS[CONFIG_ID]["seed"] + 7919 * rank


def max_over_ranks(x, world, device):
    """The slowest rank's value (the whole job's step time); identity at N=1."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank, world, seconds):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * world / seconds


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.lines = []
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "50"]
        if uuid:
            cmd += ["-i", uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def stop(self, t0, t1):
        if self.proc is None:
            return None
        time.sleep(0.12)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ts, line in self.lines:
            if not (t0 - 0.06 <= ts <= t1 + 0.06):
                continue
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ our arm
def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import __graft_entry__
    import synth
    from paper_0907_3768_gb300 import Context, _lib

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0 or world > 1:
        __graft_entry__.build() if rank == 0 else None
    if world > 1:
        dist.barrier()
        __graft_entry__.build()

    wl = synth.make_workload(CONFIG_ID, seed=shard_seed(rank))
    C, K, G = wl.n_cells_total, wl.K, wl.G
    ld = (K + 3) // 4 * 4
    Jbuf = torch.zeros((C, ld), dtype=torch.float32, device=dev)
    Jbuf[:, :K] = torch.from_numpy(wl.J).to(dev)
    J = Jbuf[:, :K]
    n = torch.from_numpy(wl.n).to(dev)
    stream = torch.cuda.current_stream(dev)

    ctxs = {}
    for p in args.paths.split(","):
        c = Context.from_workload(wl, precision=p, device=local)
        try:
            c.solve(J[:256], n[:256], precision=p)
            torch.cuda.synchronize()
            ctxs[p] = c
        except _lib.DustError as e:
            print(f"# precision {p} unavailable: {e}", file=sys.stderr)
            c.close()
    main = args.precision if args.precision in ctxs else "fp32"

    def timed(ctx, steps, warmup, prec, want_L=True, want_resid=True, profile=False, clocks=False):
        out = ctx.alloc_outputs(C, ld, want_L, want_resid, True)
        for _ in range(warmup):
            ctx.solve(J, n, precision=prec, out=out, stream=stream)
        torch.cuda.synchronize()
        nl0 = _lib.dust_ctx_launch_count(ctx.handle)
        _lib.dust_ctx_profile_read(ctx.handle)
        if profile:
            _lib.dust_ctx_profile(ctx.handle, True)
        sampler = ClockSampler(_uuid(dev)) if clocks else None
        if clocks:
            time.sleep(0.3)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(stream)
        for _ in range(steps):
            ctx.solve(J, n, precision=prec, out=out, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        if world > 1:
            dist.barrier()
        ms = max_over_ranks(e0.elapsed_time(e1) / steps, world, dev)
        launches[id(ctx), want_L, want_resid] = (_lib.dust_ctx_launch_count(ctx.handle) - nl0) / steps
        prof = None
        if profile:
            a, b, c, cnt = _lib.dust_ctx_profile_read(ctx.handle)
            _lib.dust_ctx_profile(ctx.handle, False)
            prof = (a / max(cnt, 1), b / max(cnt, 1), c / max(cnt, 1), cnt)
        clk = sampler.stop(t0, t1) if sampler else None
        return ms, out, prof, clk

    res = {}
    launches = {}
    ms_main, out_main, prof_main, clk = timed(ctxs[main], args.steps, args.warmup, main, profile=True, clocks=True)
    launches_main = launches[id(ctxs[main]), True, True]
    res[main] = dict(ms_step=ms_main, out=out_main, prof=prof_main)
    others = [p for p in ctxs if p != main]
    k2 = max(3, min(args.steps, 60))
    for p in others:
        ms, out, prof, _ = timed(ctxs[p], k2, 3, p, profile=True)
        res[p] = dict(ms_step=ms, out=out, prof=prof)
    for p in ctxs:
        ms_t, _, prof_t, _ = timed(ctxs[p], k2, 3, p, want_L=False, want_resid=False, profile=True)
        res[p]["ms_T_only"] = ms_t
        res[p]["prof_T_only"] = prof_t
    for p in res:
        ok = ctxs[p].check()
        if ok != 0:
            raise RuntimeError(f"device status {ok} after {p} runs")

    # end to end through the host-buffer entry point (pinned host memory):
    # every step copies J and n in and T, L, resid, flags out
    e2e = None
    if not args.no_e2e:
        Jh = torch.zeros((C, ld), dtype=torch.float32).pin_memory()
        Jh[:, :K] = torch.from_numpy(wl.J)
        nh = torch.from_numpy(wl.n).pin_memory()
        Th = torch.empty((C, G), dtype=torch.float32).pin_memory()
        Lh = torch.empty((C, ld), dtype=torch.float32).pin_memory()
        rh = torch.empty((C,), dtype=torch.float64).pin_memory()
        fh = torch.empty((C, G), dtype=torch.uint8).pin_memory()
        cm = ctxs[main]
        cm.set_precision(main)
        args_h = (cm.handle, C, Jh.data_ptr(), ld, nh.data_ptr(), Th.data_ptr(), Lh.data_ptr(), rh.data_ptr(),
                  fh.data_ptr())
        for _ in range(2):
            _lib.dust_solve_host(*args_h)
        ke = max(3, min(args.steps, 30))
        if world > 1:
            dist.barrier()
        tt = []
        for _ in range(ke):
            t0 = time.perf_counter()
            _lib.dust_solve_host(*args_h)
            tt.append(time.perf_counter() - t0)
        te = max_over_ranks(sum(tt) / ke, world, dev)
        h2d = C * ld * 4 + C * G * 4
        d2h = C * G * 4 + C * ld * 4 + C * 8 + C * G
        # value: the mean over the steps (whole-job throughput); the median
        # beside it shows how much of that is the host (a call is host-driven:
        # six copies and five launches per chunk)
        e2e = {"value": aggregate_rate(C * G, world, te), "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": round(te * 1e3, 4), "ms_per_step_median": round(sorted(tt)[ke // 2] * 1e3, 4),
               "api": "dust_solve_host (pinned host buffers)"}
    # time per call against the cell count (with the host entry point, so it
    # goes with the e2e leg)
    sweep = None
    if not args.no_sweep and not args.no_e2e and world == 1:
        sweep = size_sweep(ctxs[main], J, n, stream, args_h)

    # roofline of the dominant kernel: the warp-specialized solve + emission where
    # it applies (its solve is timed with the emission), else the emission kernel;
    # either way one MUFU ex2 per Planck term
    ex2_rate, fma_rate = _lib.dust_diag_throughput(local)
    ms_emit = res[main]["prof"][2]
    solve_in_emit = res[main]["prof"][1] < 0.02 * ms_emit
    terms = C * G * K
    traffic_b, traffic_note = recorded_traffic("k_solve_emit" if solve_in_emit else "k_emit")
    achieved = terms / (ms_emit * 1e-3) / 1e9
    peak = ex2_rate / 1e9
    roofline = {"bound": "alu",
                "kernel": ("k_solve_emit (temperature solve + emission + residual fold, warp-specialized)"
                           if solve_in_emit else "k_emit (emission) + k_resid"),
                "achieved": round(achieved, 2), "peak": round(peak, 2), "unit": "G Planck terms/s",
                "frac": round(achieved / peak, 4),
                "peak_source": "measured MUFU ex2.approx issue rate (dust_diag_throughput), 1 ex2 per term",
                "traffic": traffic_b if (C, K, G) == (1 << 18, 200, 96) and world == 1 else None,
                "traffic_unit": "bytes per launch (ncu DRAM read + write)",
                "traffic_source": traffic_note,
                # per cell, fused: S, n and the order index in; T, flags, L and the residual out; the cell
                # record and the k-group partials once (written, then read back by the fold).  Two-kernel
                # emission: pairs, record and order index in; L and the partials out
                "algorithmic_bytes": C * (4 * ((G + 15) // 16 * 16) + 4 * G + 4 + 4 * G + G + 4 * K + 8 + 16
                                          + 8 * ((K + 7) // 8))
                if solve_in_emit else C * (8 * ((G + 7) // 8 * 8) + 16 + 4 + 4 * K + 8 * ((K + 7) // 8)),
                "ms_per_launch": round(ms_emit, 4),
                "fma_pipe_peak_Gflop_lanes": round(fma_rate / 1e9, 1)}
    if solve_in_emit:
        # the same step with the solve and the emission as two kernels
        cm = ctxs[main]
        cm.set_fused_emit(False)
        try:
            ms_2, out_2, prof_2, _ = timed(cm, k2, 3, main, profile=True)
            same2 = all(torch.equal(out_2[k], res[main]["out"][k]) for k in ("T", "flags", "L", "resid"))
            del out_2
        finally:
            cm.set_fused_emit(True)
        roofline["emission_kernel_alone"] = {
            "kernel": "k_emit + k_resid (solve in its own kernel)", "ms_per_launch": round(prof_2[2], 4),
            "achieved": round(terms / (prof_2[2] * 1e-3) / 1e9, 2), "frac": round(terms / (prof_2[2] * 1e-3) / ex2_rate, 4),
            "step_ms": round(ms_2, 5), "ms_solve": round(prof_2[1], 5), "bitwise_equal": bool(same2)}

    # ablation of the split's third product: J split, W rounded to 16 bits once (two MMAs per K step)
    ablation_products, extra_out = None, {}
    if main != "fp32":
        cm = ctxs[main]
        cm.set_split_products(2)
        try:
            ms_p, out_p, prof_p, _ = timed(cm, k2, 3, main, profile=True)
        finally:
            cm.set_split_products(3)
        ablation_products = {"products": 2, "ms_step": round(ms_p, 5), "ms_absorb_and_order": round(prof_p[0], 5),
                             "three_products_ms_step": round(ms_main, 5),
                             "three_products_ms_absorb_and_order": round(res[main]["prof"][0], 5),
                             "note": "dust_ctx_set_split_products(ctx, 2): J_hi W_hi + J_lo W_hi, the J_hi W_lo "
                                     "product left out; not held to the mixed tolerances"}
        extra_out["two_products"] = out_p

    line = {
        "metric": METRIC, "value": aggregate_rate(C * G, world, ms_main * 1e-3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_main, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": f"{main} GEMM (16-bit hi/lo split products, f32 accumulate), f32 solve and emission"
        if main != "fp32" else "f32",
        "data": "synthetic (seeded generators: 2-temperature stellar field x U, toy grain model, MRN sizes)",
        "config": {"workload": WORKLOAD, "precision": main, "cells_per_gpu": C, "K": K, "G": G,
                   "l2": "inputs larger than L2 (J 210 MB, L 210 MB per step)",
                   "parallelism": f"dp{world} (independent cell batches)"},
        "sed_cells_per_s": C * world / (ms_main * 1e-3),
        "gpu_launches": int(round(launches_main * args.steps)),
        "roofline": roofline,
        "clocks": clk,
        "e2e": e2e,
    }
    if sweep is not None:
        line["size_sweep"] = sweep
    paths = {}
    for p in ctxs:
        r = res[p]
        paths[p] = {"ms_step": round(r["ms_step"], 5),
                    "solves_per_s": C * G * world / (r["ms_step"] * 1e-3),
                    "sed_cells_per_s": C * world / (r["ms_step"] * 1e-3),
                    "ms_absorb": round(r["prof"][0], 5), "ms_solve": round(r["prof"][1], 5),
                    "ms_emit": round(r["prof"][2], 5),
                    "solve_inside_emission_kernel": bool(r["prof"][1] < 0.02 * r["prof"][2]),
                    "T_only_ms": round(r["ms_T_only"], 5),
                    "T_only_solves_per_s": C * G * world / (r["ms_T_only"] * 1e-3)}
    line["paths"] = paths
    if main != "fp32" and not args.no_fused:
        # the same step with absorption and temperature solve as one kernel
        cm = ctxs[main]
        cm.set_fused(True)
        try:
            ms_f, out_f, prof_f, _ = timed(cm, k2, 3, main, profile=True)
            ms_ft, _, prof_ft, _ = timed(cm, k2, 3, main, want_L=False, want_resid=False, profile=True)
            same = all(torch.equal(out_f[k], res[main]["out"][k]) for k in ("T", "flags", "L"))
            del out_f
        finally:
            cm.set_fused(False)
        line["paths"][main + "_fused_absorb_solve"] = {
            "ms_step": round(ms_f, 5), "solves_per_s": aggregate_rate(C * G, world, ms_f * 1e-3),
            "ms_absorb_solve": round(prof_f[0], 5), "ms_emit": round(prof_f[2], 5),
            "T_only_ms": round(ms_ft, 5), "T_only_solves_per_s": aggregate_rate(C * G, world, ms_ft * 1e-3),
            "bitwise_equal_T_flags_L": bool(same),
            "api": "dust_ctx_set_fused(ctx, 1): k_absorb_solve (tcgen05 GEMM whose epilogue solves T), then k_emit"}
    if not args.no_mass:
        line["paths"][main + "_dust_mass_form"] = mass_form(ctxs[main], wl, J, stream, args, world, dev)
    if not args.no_ablation:
        line["ablation_paper_kernel3"] = paper_newton_ablation(ctxs[main], wl, J, stream, res[main]["ms_T_only"])
    if not args.no_coupled:
        line["coupled_self_absorption"] = coupled_solve(ctxs[main], wl, J, n, stream)

    if not args.no_fluct:
        line["fluctuating_grains"] = fluctuating(ctxs[main], wl, J, n, stream, args, world, ex2_rate,
                                                 oracle_sample=rank == 0 and world == 1 and not args.no_cpu_baseline)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"], line["err_vs_oracle"], extra_err, line["cpu_interp_baseline"] = cpu_baseline(
            args, wl, res, extra_out)
        line["cpu_interp_baseline"]["gpu_speedup"] = line["value"] / line["cpu_interp_baseline"]["value"]
        if ablation_products is not None:
            ablation_products["err_vs_oracle"] = extra_err.get("two_products")
    if ablation_products is not None:
        line["ablation_split_products"] = ablation_products
    extra_out.clear()
    del out_main, res, Jbuf, J, n
    torch.cuda.empty_cache()
    if not args.no_large:
        line["large"] = run_large(args, dev, local, ex2_rate)
        torch.cuda.empty_cache()
    if not args.no_serving:
        line["serving"] = run_serving(args, dev, local)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the error against the FP64 oracle of every workload configuration the line covers
        byc = {"0 tiny: 1024 cells x 64 wavelengths x 16 grains, all cells": tiny_errors(local, dev),
               "1-2 main: 2^18 cells x 200 x 96, first cells (as cpu_baseline)": line.get("err_vs_oracle")}
        if "large" in line:
            byc["3 large: 2^20 cells x 500 x 240, 10% near-opaque"] = line["large"].get("err_vs_oracle")
        if "serving" in line:
            byc["4 serving: Poisson stream, BF16x3 server"] = line["serving"].get("err_vs_oracle")
        line["err_by_config"] = byc
    if rank == 0:
        print(json.dumps(line), flush=True)
    for c in ctxs.values():
        c.close()
    if world > 1:
        dist.destroy_process_group()



def fluctuating(ctx, wl, J, n, stream, args, world, ex2_rate, oracle_sample):
    """Temperature distributions of the workload's 0.5-10 nm grains (36 of
    96) on M levels each, and their emission: one kernel per step over the
    same resident J.  Planck terms counted are C Gf (M - 1) K; the oracle of
    the same method is timed on a bounded sample of cells."""
    import time

    import numpy as np
    import torch

    import synth
    from synth.workloads import heat_capacity_params

    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from metrics import l_err

    grains = synth.fluctuating_selection(wl.a_of_g)
    N, th = heat_capacity_params(synth.CONFIGS[1]["species"], wl.sp_of_g, wl.a_of_g)
    M = args.fluct_levels
    ctx.set_fluctuating(grains, N[grains], th[grains], M)
    C, K, Gf = J.shape[0], ctx.K, len(grains)
    n_f = n[:, torch.from_numpy(grains).to(n.device)].contiguous()
    out = ctx.solve_fluct(J, n_f, want_dE=False, stream=stream)
    for _ in range(max(3, args.warmup) - 1):
        ctx.solve_fluct(J, n_f, want_dE=False, out=out, stream=stream)
    torch.cuda.synchronize()
    steps = max(3, min(args.steps, 10))
    l0 = _lib_launches(ctx)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        ctx.solve_fluct(J, n_f, want_dE=False, out=out, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    launches = (_lib_launches(ctx) - l0) / steps
    assert ctx.check() == 0
    terms = C * Gf * (M - 1) * K
    fl_traffic, fl_note = recorded_traffic("k_fluct")
    r = {"workload": f"{C} cells x {K} wavelengths; {Gf} fluctuating grains of 0.5-10 nm (Einstein enthalpy) "
                     f"x {M} levels; inputs resident in HBM",
         "method": "per (cell, grain): level grid from the equilibrium T, photon-bin heating rates by two prefix "
                   "sums, thermal-continuous cooling from the P_g table, cut-flux recursion, ex2 emission (FP32)",
         "ms_per_step": round(ms, 3), "distributions_per_s": aggregate_rate(C * Gf, world, ms * 1e-3),
         "planck_terms_per_s": aggregate_rate(terms, world, ms * 1e-3), "launches_per_step": launches,
         "roofline": {"kernel": "k_fluct", "bound": "alu", "unit": "G Planck terms/s",
                      "achieved": round(terms / (ms * 1e-3) / 1e9, 1), "peak": round(ex2_rate / 1e9, 1),
                      "frac": round(terms / (ms * 1e-3) / ex2_rate, 4),
                      "peak_source": "measured MUFU ex2.approx rate (dust_diag_throughput)",
                      "traffic": fl_traffic if M == 128 and K == 200 and fl_traffic is not None else None,
                      "traffic_source": fl_note,
                      "algorithmic_bytes": C * (2 * K + Gf) * 4}}
    if oracle_sample:
        from oracle import fluct as ofl

        cells = np.array([0, C // 3, (2 * C) // 3])[: max(1, min(3, C))]
        t0 = time.perf_counter()
        ref = ofl.run(wl.lam, wl.w, wl.C_abs, wl.J[cells], wl.n[cells][:, grains], grains, N[grains], th[grains], M,
                      wl.T_min, wl.T_max, want_P=True)
        sec = time.perf_counter() - t0
        o = ctx.solve_fluct(J[torch.from_numpy(cells).to(J.device)], n_f[torch.from_numpy(cells).to(J.device)],
                            want_P=True, stream=stream)
        torch.cuda.synchronize()
        P = o["P"].cpu().numpy()
        r["cpu_baseline"] = {"value": len(cells) * Gf / sec, "unit": "distributions/s", "cores": 1, "kind": "oracle",
                             "sample": f"{len(cells)} cells x {Gf} grains x {M} levels (FP64 numpy, "
                                       "transition matrix built one photon landing at a time)"}
        r["err_vs_oracle"] = {"L_max": float(l_err(o["L"][:, :K].cpu().numpy(), ref["L"]).max()),
                              "P_max_abs_over_peak": float((np.abs(P - ref["P"]) /
                                                            ref["P"].max(axis=2, keepdims=True)).max()),
                              "cells": len(cells)}
    del out
    return r


def _lib_launches(ctx):
    from paper_0907_3768_gb300 import _lib

    return _lib.dust_ctx_launch_count(ctx.handle)


def paper_newton_ablation(ctx, wl, J, stream, ms_table_T_only):
    """The paper's own temperature method (per-iterate quadrature Newton from
    the Eqs. 11-12 guess, 0.1 % stop) on the same cells and the same GEMM,
    against the table solve's temperature-only step."""
    import torch

    ctx.set_grain_sizes(wl.a_of_g)
    C, G = J.shape[0], ctx.G
    for _ in range(2):
        out = ctx.solve_T_newton(J, stream=stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 3
    e0.record(stream)
    for _ in range(reps):
        out = ctx.solve_T_newton(J, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    it = out["iters"][out["flags"] == 0].float()
    return {"ms_per_step": round(ms, 4), "solves_per_s": C * G / (ms * 1e-3),
            "table_T_only_ms": round(ms_table_T_only, 4),
            "table_speedup": round(ms / ms_table_T_only, 1),
            "newton_steps_mean": round(float(it.mean()), 3), "newton_steps_max": int(it.max()),
            "not_converged": int((out["flags"] == 8).sum()),
            "method": "per (cell, grain) Newton in T with the K-term quadrature at every iterate, "
                      "Eqs. 11-12 guess floored at 5 K, stop at 0.1 % energy non-conservation; same BF16x3 GEMM"}


def mass_form(ctx, wl, J, stream, args, world, dev):
    """The same step through dust_solve_mass: the workload's grain numbers are
    n[c,g] = rho_c n0_g, so n_g = n[0,:] and m_c = n[c,0] / n[0,0]."""
    import numpy as np
    import torch

    n64 = wl.n.astype(np.float64)
    ctx.set_grain_numbers(n64[0])
    m = torch.from_numpy((n64[:, 0] / n64[0, 0]).astype(np.float32)).to(dev)
    C, G = J.shape[0], ctx.G
    out = ctx.alloc_outputs(C, J.stride(0))
    for _ in range(max(3, args.warmup)):
        ctx.solve_mass(J, m, out=out, stream=stream)
    torch.cuda.synchronize()
    steps = max(3, min(args.steps, 60))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        ctx.solve_mass(J, m, out=out, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1) / steps, world, dev)
    return {"ms_step": round(ms, 5), "solves_per_s": aggregate_rate(C * G, world, ms * 1e-3),
            "sed_cells_per_s": aggregate_rate(C, world, ms * 1e-3),
            "api": "dust_solve_mass (n[c,g] = n_g m_c, Eqs. 9-10)"}


def coupled_solve(ctx, wl, J, n, stream):
    """The self-absorbing iteration J = J_ext + E L on the same cells, with a
    coupling that returns a fraction f_c ~ U(0, 0.5) of each cell's absorbed
    power as its own re-absorbed emission: E = f_c / (4 pi sum_g n C)."""
    import math

    import numpy as np
    import torch

    f = np.random.default_rng(4244).uniform(0.0, 0.5, wl.n_cells_total)
    kappa = torch.from_numpy(wl.n).to(J.device).double() @ torch.from_numpy(wl.C_abs).to(J.device)
    Eb = torch.zeros_like(J.as_strided((J.shape[0], J.stride(0)), (J.stride(0), 1)))
    Eb[:, :wl.K] = (torch.from_numpy(f).to(J.device)[:, None] / (4.0 * math.pi * kappa)).float()
    E = Eb[:, :wl.K]
    del kappa
    ctx.solve_coupled(J[:4096], E[:4096], n[:4096], max_iters=3, tol=0.0, stream=stream)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out, it, ch = ctx.solve_coupled(J, E, n, max_iters=100, tol=1e-6, stream=stream)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    C, G = J.shape[0], ctx.G
    return {"iterations": it, "last_change": ch, "ms_total": round(dt * 1e3, 3),
            "ms_per_iteration": round(dt * 1e3 / it, 4), "solves_per_s": C * G * it / dt,
            "coupling": "E = f_c / (4 pi sum_g n C), f_c ~ U(0, 0.5); stop at 1e-6 peak-normalised change of L"}


def _uuid(dev):
    import torch

    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return None


def _oracle_sample(seconds, cfg_id=CONFIG_ID, seed=None):
    """Oracle on the first cells of the workload, sized to ~`seconds` of work."""
    import numpy as np

    import oracle
    import synth

    probe = synth.make_workload(cfg_id, cells=np.arange(64), seed=seed)
    t = time.perf_counter()
    oracle.run_workload(probe)
    per_cell = (time.perf_counter() - t) / 64
    ncell = int(max(64, min(synth.CONFIGS[cfg_id]["n_cells"], seconds / max(per_cell, 1e-9))))
    wl = synth.make_workload(cfg_id, cells=np.arange(ncell), seed=seed)
    t = time.perf_counter()
    ref = oracle.run_workload(wl)
    dt = time.perf_counter() - t
    return wl, ref, dt, oracle.max_threads()


def tiny_errors(local, dev):
    """The 1024-cell, 64-wavelength, 16-grain case in every precision against the oracle, in full."""
    import numpy as np
    import torch

    import oracle
    import synth
    from paper_0907_3768_gb300 import Context, padded_rows

    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from metrics import l_err, t_err

    wl = synth.make_workload(0)
    ref = oracle.run_workload(wl)
    J = padded_rows(torch.from_numpy(wl.J).to(dev))
    n = torch.from_numpy(wl.n).to(dev)
    errs = {"cells": len(wl.cells)}
    for prec in ("fp32", "bf16x3", "fp16x3"):
        with Context.from_workload(wl, precision=prec, device=local) as ctx:
            o = ctx.solve(J, n)
            torch.cuda.synchronize()
            assert ctx.check() == 0
            T, L = o["T"].cpu().numpy(), o["L"].cpu().numpy()[:, :wl.K]
            fl, rs = o["flags"].cpu().numpy(), o["resid"].cpu().numpy()
        eT, eL = t_err(T, ref["T"], ref["flags"]), l_err(L, ref["L"])
        ok = (ref["flags"] == 0).all(axis=1)
        errs[prec] = {"T_max": float(eT.max()), "T_p99": float(np.percentile(eT, 99)), "L_max": float(eL.max()),
                      "L_p99": float(np.percentile(eL, 99)), "resid_max": float(np.abs(rs[ok]).max(initial=0.0)),
                      "flags_equal": bool((fl == ref["flags"]).all())}
    return errs


def cpu_baseline(args, wl_full, res, extra=None):
    import numpy as np

    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from metrics import l_err, t_err

    wl, ref, dt, cores = _oracle_sample(args.cpu_seconds, seed=wl_full.seed)
    nc = len(wl.cells)
    base = {"value": nc * wl.G / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {nc} of {wl_full.n_cells_total} cells, full path (A, Brent T, L, resid), "
                      f"FP64 C + OpenMP, {dt:.1f} s"}
    errs = {}
    items = [(p, r["out"], errs) for p, r in res.items()]
    extra_errs = {}
    items += [(p, o, extra_errs) for p, o in (extra or {}).items()]
    for p, out, dst in items:
        T = out["T"][:nc].cpu().numpy()
        L = out["L"][:nc].cpu().numpy()
        fl = out["flags"][:nc].cpu().numpy()
        rs = out["resid"][:nc].cpu().numpy()
        eT = t_err(T, ref["T"], ref["flags"])
        eL = l_err(L, ref["L"])
        dst[p] = {"T_max": float(eT.max()), "T_p99": float(np.percentile(eT, 99)),
                  "L_max": float(eL.max()), "L_p99": float(np.percentile(eL, 99)),
                  "resid_max": float(np.abs(rs).max()), "flags_equal": bool((fl == ref["flags"]).all()),
                  "cells": nc}
    return base, errs, extra_errs, cpu_interp_baseline(args, wl_full, wl, ref)


def cpu_interp_baseline(args, wl_full, wl_o, ref):
    """The paper's CPU production scheme (Section 6, Table 1's "CPU
    (interpolation)" column): A in full, T from a 2000-point table over
    3-1500 K, L in full, FP64 on every host core.  Timed on the first cells of
    the workload (about --cpu-interp-seconds of work; the table build is not
    timed); its error against the oracle on the oracle's sample cells."""
    import numpy as np

    import synth
    from metrics import l_err, t_err
    from oracle import cpu_interp

    t = time.perf_counter()
    tab = cpu_interp.for_workload(wl_o)
    t_tab = time.perf_counter() - t
    r = tab.run(wl_o.J, wl_o.n)
    eT = t_err(r["T"], ref["T"], ref["flags"])
    eL = l_err(r["L"], ref["L"])
    errs = {"T_max": float(eT.max()), "T_p99": float(np.percentile(eT, 99)), "L_max": float(eL.max()),
            "L_p99": float(np.percentile(eL, 99)), "flags_equal": bool((r["flags"] == ref["flags"]).all()),
            "cells": len(wl_o.cells)}
    probe = synth.make_workload(CONFIG_ID, cells=np.arange(512), seed=wl_full.seed)
    t = time.perf_counter()
    tab.run(probe.J, probe.n)
    per_cell = (time.perf_counter() - t) / 512
    nc = int(max(512, min(wl_full.n_cells_total, args.cpu_interp_seconds / max(per_cell, 1e-9))))
    wl = synth.make_workload(CONFIG_ID, cells=np.arange(nc), seed=wl_full.seed)
    t = time.perf_counter()
    tab.run(wl.J, wl.n)
    dt = time.perf_counter() - t
    from oracle import max_threads

    return {"value": nc * wl.G / dt, "unit": UNIT, "cells_per_s": nc / dt, "cores": max_threads(),
            "kind": "paper's CPU interpolation scheme",
            "sample": f"first {nc} of {wl_full.n_cells_total} cells: A (Eq. 6), T from a 2000-point table "
                      f"over 3-1500 K (uniform in ln T, linear in P), L (Eq. 10); FP64 C + OpenMP, {dt:.1f} s "
                      f"(table build {t_tab:.2f} s, not timed)",
            "err_vs_oracle": errs}


def size_sweep(ctx, J, n, stream, args_h):
    """Time per call against the number of cells, from 32 to 2^19 (the cell
    counts of the paper's Table 1): dust_solve on device buffers (CUDA events,
    the full path with L, resid and flags) and, up to the resident workload's
    size, dust_solve_host from pinned host buffers (wall clock, copies
    included, the median of single calls).  Below ~2^16 cells the inputs stay
    in L2: a latency sweep, not a bandwidth one.  2^19 cells repeat the
    2^18-cell workload twice."""
    import numpy as np
    import torch

    from paper_0907_3768_gb300 import _lib

    C = J.shape[0]
    J2, n2 = torch.cat([J, J]), torch.cat([n, n])
    rows = []
    for Cs in (32, 256, 2048, 16384, 131072, 262144, 524288):
        if Cs > 2 * C:
            break
        Js, ns = (J2, n2) if Cs > C else (J, n)
        Js, ns = Js[:Cs], ns[:Cs]
        out = ctx.solve(Js, ns, stream=stream)
        for _ in range(2):
            ctx.solve(Js, ns, out=out, stream=stream)
        reps = max(5, min(200, int(2e6 // Cs)))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        t0 = time.perf_counter()
        for _ in range(reps):
            ctx.solve(Js, ns, out=out, stream=stream)
        t_issue = (time.perf_counter() - t0) / reps
        e1.record(stream)
        torch.cuda.synchronize()
        ms_dev = e0.elapsed_time(e1) / reps
        # host time to issue one call (Python binding, argument checks, five
        # launches): where it matches ms_device the device waited on the host
        row = {"cells": Cs, "ms_device": round(ms_dev, 4), "cells_per_s_device": round(Cs / (ms_dev * 1e-3)),
               "ms_host_issue": round(t_issue * 1e3, 4)}
        if args_h is not None and Cs <= C:
            a = list(args_h)
            a[1] = Cs
            for _ in range(2):
                _lib.dust_solve_host(*a)
            # the median of single calls: a call is host-driven (six copies and
            # five launches per chunk), so one descheduled host thread would
            # otherwise move a mean over a few calls
            tt = []
            for _ in range(max(7, min(100, int(5e5 // Cs)))):
                t0 = time.perf_counter()
                _lib.dust_solve_host(*a)
                tt.append(time.perf_counter() - t0)
            ms_h = float(np.median(tt)) * 1e3
            row.update({"ms_host": round(ms_h, 4), "cells_per_s_host": round(Cs / (ms_h * 1e-3))})
        rows.append(row)
    assert ctx.check() == 0
    del J2, n2
    return {"api": "dust_solve (device buffers, CUDA events) and dust_solve_host (pinned host buffers, wall clock)",
            "precision": "bf16x3", "rows": rows}


# ------------------------------------------------------------------ large solve
def run_large(args, dev, local, ex2_rate):
    """The 2^20-cell, 500-wavelength, 240-grain solve (10 % near-opaque cells):
    full-path and temperature-only times per precision, with the per-kernel
    split and the rooflines of both kernels."""
    import json as _json  # noqa: F401
    import torch

    import synth
    from paper_0907_3768_gb300 import Context, _lib

    import numpy as np

    full = synth.CONFIGS[3]["n_cells"]
    wl = synth.make_workload(3, cells=None if args.large_cells >= full else np.arange(args.large_cells))
    C, K, G = len(wl.cells), wl.K, wl.G
    ld = (K + 3) // 4 * 4
    Jb = torch.zeros((C, ld), dtype=torch.float32, device=dev)
    Jb[:, :K] = torch.from_numpy(wl.J).to(dev)
    J, n = Jb[:, :K], torch.from_numpy(wl.n).to(dev)
    del wl
    stream = torch.cuda.current_stream(dev)
    out = {"workload": f"{C} cells x 500 wavelengths (0.05-2000 um) x 240 grains, 10% near-opaque cells"}
    steps = max(3, min(args.steps, 10))
    # error sample: every (C // 128)-th cell and the first 32 near-opaque cells
    from synth.workloads import _cell_draws

    opaque = np.nonzero(_cell_draws(synth.CONFIGS[3], full, synth.CONFIGS[3]["seed"])[2][:C])[0][:32]
    sample = np.unique(np.concatenate([np.arange(0, C, max(1, C // 128)), opaque]))
    kept = {}
    for prec in ("bf16x3", "fp32"):
        ctx = Context.from_workload(synth.make_workload(3, cells=[0]), precision=prec, device=local)
        r = {}
        for mode, wantL in (("full", True), ("T_only", False)):
            o = ctx.alloc_outputs(C, ld, wantL, wantL, True)
            for _ in range(2):
                ctx.solve(J, n, out=o, stream=stream)
            torch.cuda.synchronize()
            _lib.dust_ctx_profile_read(ctx.handle)
            _lib.dust_ctx_profile(ctx.handle, True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                ctx.solve(J, n, out=o, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            a, b, c, cnt = _lib.dust_ctx_profile_read(ctx.handle)
            _lib.dust_ctx_profile(ctx.handle, False)
            ms = e0.elapsed_time(e1) / steps
            r[mode] = {"ms_step": round(ms, 4), "ms_absorb": round(a / cnt, 4), "ms_solve": round(b / cnt, 4),
                       "ms_emit": round(c / cnt, 4),
                       "solves_per_s": C * G / (ms * 1e-3), "sed_cells_per_s": C / (ms * 1e-3) if wantL else None}
            if wantL:
                idx = torch.from_numpy(sample).to(dev)
                kept[prec] = {k: o[k][idx].cpu().numpy() for k in ("T", "L", "flags", "resid")}
            del o
        if prec != "fp32":
            # the split's third product left out (an ablation): the GEMM is near its tensor bound here
            ctx.set_split_products(2)
            o = ctx.alloc_outputs(C, ld, False, False, True)
            for _ in range(2):
                ctx.solve(J, n, out=o, stream=stream)
            torch.cuda.synchronize()
            _lib.dust_ctx_profile_read(ctx.handle)
            _lib.dust_ctx_profile(ctx.handle, True)
            for _ in range(steps):
                ctx.solve(J, n, out=o, stream=stream)
            torch.cuda.synchronize()
            a, b, c, cnt = _lib.dust_ctx_profile_read(ctx.handle)
            _lib.dust_ctx_profile(ctx.handle, False)
            ctx.set_split_products(3)
            del o
            r["T_only_two_products"] = {"ms_absorb": round(a / cnt, 4), "ms_solve": round(b / cnt, 4),
                                        "note": "dust_ctx_set_split_products(ctx, 2), temperatures only"}
        assert ctx.check() == 0
        ctx.close()
        ms_a, ms_b = r["full"]["ms_absorb"], r["full"]["ms_emit"]
        r["roofline_emit"] = {"bound": "alu", "unit": "G Planck terms/s",
                              "kernels": "k_solve_emit (temperature solve + first grain pass) + k_emit (later passes)"
                                         " + k_resid" if r["full"]["ms_solve"] < 0.02 * ms_b else "k_emit + k_resid",
                                    "achieved": round(C * G * K / (ms_b * 1e-3) / 1e9, 1),
                                    "peak": round(ex2_rate / 1e9, 1),
                                    "frac": round(C * G * K / (ms_b * 1e-3) / ex2_rate, 4)}
        gbytes = (C * K * 4 + C * ((G + 15) // 16 * 16) * 4) / 1e9
        r["roofline_absorb"] = {"bound": "hbm", "unit": "GB/s", "achieved": round(gbytes / (ms_a * 1e-3), 1),
                                "peak": HBM_PEAK, "frac": round(gbytes / (ms_a * 1e-3) / HBM_PEAK, 4),
                                "peak_source": HBM_PEAK_SOURCE,
                                "tensor_TFLOPs_executed": round((3 if prec != "fp32" else 1) * 2 * C * G * K /
                                                                (ms_a * 1e-3) / 1e12, 1)}
        if prec != "fp32":
            # the three 16-bit products on the tensor pipe against the dense BF16 peaks (FP16 runs at
            # the same rate); the GEMM runs inside a 25 ms step, so the sustained figure applies
            tf = r["roofline_absorb"]["tensor_TFLOPs_executed"]
            r["roofline_absorb"]["tensor_frac_of_sustained_bf16"] = round(tf / BF16_SUSTAINED, 4)
            r["roofline_absorb"]["tensor_frac_of_burst_bf16"] = round(tf / BF16_BURST, 4)
            r["roofline_absorb"]["tensor_peak_source"] = BF16_SOURCE
        out[prec] = r
    # error against the oracle on the sample
    import oracle

    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from metrics import l_err, t_err

    ws = synth.make_workload(3, cells=sample)
    t0 = time.perf_counter()
    ref = oracle.run_workload(ws)
    dt = time.perf_counter() - t0
    errs = {}
    for prec, k in kept.items():
        eT = t_err(k["T"], ref["T"], ref["flags"])
        eL = l_err(k["L"][:, :K], ref["L"])
        ok = (ref["flags"] == 0).all(axis=1)
        errs[prec] = {"T_max": float(eT.max()), "T_p99": float(np.percentile(eT, 99)), "L_max": float(eL.max()),
                      "L_p99": float(np.percentile(eL, 99)), "resid_max": float(np.abs(k["resid"][ok]).max(initial=0.0)),
                      "flags_equal": bool((k["flags"] == ref["flags"]).all())}
    out["err_vs_oracle"] = dict(errs, sample=f"{len(sample)} cells: every {max(1, C // 128)}-th and the first "
                                              f"{len(opaque)} near-opaque ones; oracle {dt:.1f} s")
    return out


# ------------------------------------------------------------------ serving
def run_serving(args, dev, local):
    """Request stream shaped like the serving workload: Poisson arrivals of
    solves from 64 snapshots, cells log-uniform 1e3-1e6, K in {100, 200, 350,
    500}, G in {48, 96, 240}.  The inputs of every (K, G) grid are generated
    once, before any timing, into one resident buffer as large as the grid's
    largest request (same recipe as synth, seeded per grid); a request solves a
    seeded slice of its grid's buffer, so the timed loops measure the server,
    not the input generator.  Measures the saturated throughput with a closed
    loop, then a Poisson stream at `serve_load` x that rate through the
    continuous-batching server (BF16x3), and the same stream through a
    one-request-at-a-time FP32 loop."""
    import numpy as np
    import torch

    import synth
    from paper_0907_3768_gb300 import Context, Server
    from synth import workloads as W

    reqs = W.serve_requests(n_requests=args.serve_requests, rate_hz=1.0)
    cmax = {}
    for r in reqs:
        cmax[(r["K"], r["G"])] = max(cmax.get((r["K"], r["G"]), 0), r["n_cells"])
    grids = {}
    for (K, G), C in cmax.items():
        cfg = W.serve_snapshot_config(0, K, G, 8)
        wl = synth.make_workload(cfg, cells=np.arange(1))
        ld = (K + 3) // 4 * 4
        gen = torch.Generator(device=dev)
        gen.manual_seed(cfg["seed"] * 1000003 + K * 1009 + G)
        lo, hi = cfg["log10U"]
        U = 10.0 ** (torch.rand(C, generator=gen, device=dev, dtype=torch.float64) * (hi - lo) + lo)
        rho = torch.exp(torch.randn(C, generator=gen, device=dev, dtype=torch.float64))
        op = torch.rand(C, generator=gen, device=dev, dtype=torch.float64) < cfg["opaque_frac"]
        tau = torch.rand(C, generator=gen, device=dev, dtype=torch.float64) * (cfg["tau_V"][1] - cfg["tau_V"][0]) \
            + cfg["tau_V"][0]
        shape = torch.tensor(W.J_ISRF * W.stellar_shape(wl.lam), device=dev, dtype=torch.float64)
        ext = torch.tensor((wl.lam / (0.55 * W.UM)) ** -1.3, device=dev, dtype=torch.float64)
        n0 = torch.tensor(W.size_weights(wl.sp_of_g, wl.a_of_g), device=dev, dtype=torch.float64)
        Jb = torch.zeros((C, ld), dtype=torch.float32, device=dev)
        att = torch.where(op[:, None], torch.exp(-(tau[:, None] * ext[None, :])), torch.ones_like(ext)[None, :])
        Jb[:, :K] = (U[:, None] * shape[None, :] * att).float()
        del att
        grids[(K, G)] = dict(J=Jb[:, :K], n=(rho[:, None] * n0[None, :]).float().contiguous(), C=C, wl=wl,
                             mixed=Context.from_workload(wl, precision="bf16x3", device=local),
                             fp32=Context.from_workload(wl, precision="fp32", device=local))
    torch.cuda.synchronize()
    offs = np.random.default_rng(4243).random(len(reqs))

    def inputs(i):
        r = reqs[i]
        g = grids[(r["K"], r["G"])]
        C = r["n_cells"]
        o = int(offs[i] * (g["C"] - C + 1))
        return g, g["J"][o:o + C], g["n"][o:o + C]

    total_cells = sum(r["n_cells"] for r in reqs)
    total_solves = sum(r["n_cells"] * r["G"] for r in reqs)
    budget = 48 << 30
    res = {"requests": len(reqs), "cells": total_cells, "hbm_budget_bytes": budget,
           "workload": "Poisson stream, 64 snapshots, cells log-uniform 1e3-1e6, K in {100,200,350,500}, "
                       "G in {48,96,240}"}
    # closed loop: saturated throughput of the server
    with Server(budget, max_inflight=24, device=local) as srv:
        pend = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(len(reqs)):
            g, J, n = inputs(i)
            pend.append((g["mixed"].submit(srv, J, n), J, n))
            while len(pend) > 32:
                (t, _), _, _ = pend.pop(0)
                srv.wait(t, 600000.0)
        for (t, _), _, _ in pend:
            srv.wait(t, 600000.0)
        sat = time.perf_counter() - t0
        st = srv.stats()
    res["saturated"] = {"s": sat, "requests_per_s": len(reqs) / sat, "cells_per_s": total_cells / sat,
                        "solves_per_s": total_solves / sat, "rounds": st["rounds"], "launches": st["launches"]}
    # the same requests one after another through dust_solve on one stream (BF16x3, no arrival
    # pacing): the plain loop the server's batching is measured against
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(len(reqs)):
        g, J, n = inputs(i)
        out = g["mixed"].solve(J, n)
        del out
    torch.cuda.synchronize()
    b2b = time.perf_counter() - t0
    res["back_to_back_dust_solve"] = {"s": b2b, "requests_per_s": len(reqs) / b2b, "solves_per_s": total_solves / b2b,
                                      "note": "every request through dust_solve in turn on one stream, BF16x3"}
    rate = args.serve_load * len(reqs) / sat
    arrivals = np.array([r["t"] for r in reqs]) / rate
    res["rate_hz"] = rate
    res["load"] = args.serve_load

    # the first request of every (K, G) grid is kept for the error against the oracle
    keep = {}
    for i, r in enumerate(reqs):
        keep.setdefault((r["K"], r["G"]), i)
    keep = set(keep.values())

    # Poisson stream through the server
    lat_srv = np.zeros(len(reqs))
    kept = {}
    with Server(budget, max_inflight=24, device=local) as srv:
        pend, lag = {}, []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(len(reqs)):
            while time.perf_counter() - t0 < arrivals[i]:
                for t in list(pend):
                    state, ms = srv.poll(t)
                    if state in ("done", "cancelled"):
                        lat_srv[pend[t][0]] = ms
                        del pend[t]
                time.sleep(0.0002)
            lag.append(time.perf_counter() - t0 - arrivals[i])
            g, J, n = inputs(i)
            t, out = g["mixed"].submit(srv, J, n)
            pend[t] = (i, J, n, out)
            if i in keep:
                kept[i] = (g, J, n, out)
        for t in list(pend):
            state, ms = srv.poll(t)
            if state not in ("done", "cancelled"):
                ms = srv.wait(t, 600000.0)
            lat_srv[pend[t][0]] = ms
        span = time.perf_counter() - t0
        st = srv.stats()
    res["mixed_server"] = {"p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "max_ms": st["max_ms"],
                           "mean_ms": st["mean_ms"], "span_s": span, "requests_per_s": len(reqs) / span,
                           "cells_per_s": total_cells / span, "solves_per_s": total_solves / span,
                           "rounds": st["rounds"], "completed": st["completed"],
                           "client_lag_p99_ms": float(np.percentile(lag, 99) * 1e3),
                           "latency": "submit to completion, server clock",
                           "by_cells_decade": _by_decade(reqs, lat_srv)}
    res["err_vs_oracle"] = _serving_errors(kept)
    del kept

    # the same stream, one request at a time, FP32
    lat = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(len(reqs)):
        while time.perf_counter() - t0 < arrivals[i]:
            time.sleep(0.0002)
        g, J, n = inputs(i)
        out = g["fp32"].solve(J, n)
        torch.cuda.synchronize()
        lat.append((time.perf_counter() - t0 - arrivals[i]) * 1e3)
        del out
    span = time.perf_counter() - t0
    res["fp32_one_at_a_time"] = {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                                 "max_ms": float(max(lat)), "span_s": span, "requests_per_s": len(reqs) / span,
                                 "solves_per_s": total_solves / span,
                                 "latency": "arrival to completion (includes queueing behind earlier requests)",
                                 "by_cells_decade": _by_decade(reqs, np.array(lat))}
    for g in grids.values():
        g["mixed"].close()
        g["fp32"].close()
    return res


def _by_decade(reqs, lat_ms):
    """p50 / p99 latency (ms) of the requests in each decade of cell count."""
    import numpy as np

    cells = np.array([r["n_cells"] for r in reqs])
    out = {}
    for lo in (1e3, 1e4, 1e5):
        m = (cells >= lo) & (cells < lo * 10)
        if m.any():
            out[f"{int(lo):d}-{int(lo * 10):d} cells"] = {"requests": int(m.sum()),
                                                        "p50_ms": float(np.percentile(lat_ms[m], 50)),
                                                        "p99_ms": float(np.percentile(lat_ms[m], 99))}
    return out


def _serving_errors(kept, ncells=16):
    """T and L of sampled cells of the kept requests (one per grid) against the oracle."""
    import numpy as np

    import oracle

    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from metrics import l_err, t_err

    worst = {"T_max": 0.0, "L_max": 0.0, "flags_equal": True, "requests": 0, "cells": 0}
    for i, (g, J, n, out) in sorted(kept.items()):
        wl = g["wl"]
        C = J.shape[0]
        cells = np.unique(np.linspace(0, C - 1, min(ncells, C)).astype(np.int64))
        idx = torch_index(cells, J.device)
        Jh = J[idx].double().cpu().numpy()
        nh = n[idx].double().cpu().numpy()
        ref = oracle.run(wl.lam, wl.w, wl.C_abs, Jh, nh, wl.T_min, wl.T_max)
        T = out["T"][idx].cpu().numpy()
        L = out["L"][idx].cpu().numpy()[:, :wl.K]
        te = t_err(T, ref["T"], ref["flags"])
        worst["T_max"] = max(worst["T_max"], float(te.max()) if te.size else 0.0)
        worst["L_max"] = max(worst["L_max"], float(l_err(L, ref["L"]).max()))
        worst["flags_equal"] = worst["flags_equal"] and bool((out["flags"][idx].cpu().numpy() == ref["flags"]).all())
        worst["requests"] += 1
        worst["cells"] += len(cells)
    worst["sample"] = f"{ncells} cells of the first request of each (K, G) grid, BF16x3 server outputs"
    return worst


def torch_index(cells, device):
    import torch

    return torch.from_numpy(cells).to(device)


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    """The FP64 CPU oracle on the host cores (a deliberately slow baseline)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import numpy as np

    import oracle
    import synth

    oracle.lib()
    # a bounded sample per step: the whole run stays within ~100 s of CPU time
    per_step = max(0.05, min(args.cpu_seconds, 100.0 / max(1, args.steps + args.warmup)))
    wl = synth.make_workload(CONFIG_ID, cells=np.arange(64))
    t = time.perf_counter()
    oracle.run_workload(wl)
    per_cell = (time.perf_counter() - t) / 64
    ncell = int(max(8, min(4096, per_step / max(per_cell, 1e-9))))
    wl = synth.make_workload(CONFIG_ID, cells=np.arange(ncell))
    for _ in range(args.warmup):
        oracle.run_workload(wl)
    t = time.perf_counter()
    for _ in range(args.steps):
        oracle.run_workload(wl)
    dt = (time.perf_counter() - t) / args.steps
    v = ncell * wl.G / dt
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "sample_cells_per_step": ncell},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
                             "sample": f"first {ncell} cells per step, full path"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def profile_case(args):
    """Run one case's solves with nothing else on the GPU, for a profiler's launch filter."""
    import numpy as np
    import torch

    import synth
    from paper_0907_3768_gb300 import Context, padded_rows
    from synth.workloads import heat_capacity_params

    dev = torch.device("cuda", 0)
    if args.profile_case in ("main", "main-two-kernel"):
        wl = synth.make_workload(CONFIG_ID)
    elif args.profile_case == "large":
        wl = synth.make_workload(3, cells=np.arange(min(args.large_cells, synth.CONFIGS[3]["n_cells"])))
    else:
        wl = synth.make_workload(CONFIG_ID, cells=np.arange(args.profile_cells))
    J = padded_rows(torch.from_numpy(wl.J).to(dev))
    n = torch.from_numpy(wl.n).to(dev)
    with Context.from_workload(wl, precision="bf16x3") as ctx:
        if args.profile_case == "fluct":
            g = synth.fluctuating_selection(wl.a_of_g)
            N, th = heat_capacity_params(synth.CONFIGS[CONFIG_ID]["species"], wl.sp_of_g, wl.a_of_g)
            ctx.set_fluctuating(g, N[g], th[g], 128)
            nf = n[:, torch.from_numpy(g).to(dev)].contiguous()
            out = ctx.solve_fluct(J, nf, want_dE=False)
            for _ in range(args.steps):
                ctx.solve_fluct(J, nf, want_dE=False, out=out)
        else:
            ctx.set_fused_emit(args.profile_case != "main-two-kernel")
            out = ctx.solve(J, n)
            for _ in range(args.steps):
                ctx.solve(J, n, out=out)
        torch.cuda.synchronize()
        assert ctx.check() == 0
    print(json.dumps({"profile_case": args.profile_case, "cells": len(wl.cells), "K": wl.K, "G": wl.G,
                      "solves": args.steps + 1}))


def main():
    args = parse()
    if args.profile_case:
        profile_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
