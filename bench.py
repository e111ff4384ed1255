#!/usr/bin/env python
"""Throughput of the AWRTRD hot path on one GB300 (or N independent replicas).

A step is one outer iteration of Algorithm 1 (every core updated once: residuals, HQ
weights, weighted gradient, FGMC Gram, Cholesky-scaled step with exact line search) on the
100^4 workload: TR ranks 8, 50 % missing, 20 % of observed entries replaced by outliers
U[-10 std, 10 std], additive N(0, 1e-3) noise, full-tensor gradient (no sketch).  Inputs are
synthetic (seeded), the tensor (400 MB) is larger than L2, so no flush is needed between
steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16|fp32|fp64]
  python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores

Prints one JSON line on rank 0.  Besides the headline step it carries (rank 0, N = 1) the
FP32 / TF32 x 3 comparison legs, the image-shaped PSNR runs, the 1920 x 1080 x 3 x 50
completion at the paper's video rank [80, 80, 3, 20] (`video_rank80`), the other benchmark
configurations and the CPU oracle baseline; `--no-image`, `--no-video-rank80`, `--no-configs`
and `--no-cpu-baseline` skip them.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "AWRTRD iters/s & sampled entries/s to rel-err≤1e-3: BF16-TC vs FP32 on one GB300"
UNIT = "sampled entries/s"
WORKLOAD = "cfg100"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# CPU-oracle sample: the sub-tensor i_4 < 10 of the 100^4 workload (10^7 slots)
ORACLE_SLICES = 10


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default=None, choices=[None, "bf16", "tf32x3", "fp32", "fp64"])
    ap.add_argument("--no-converge", action="store_true")
    ap.add_argument("--no-image", action="store_true", help="skip the image-shaped PSNR runs")
    ap.add_argument("--image-only", action="store_true",
                    help="run only the image-shaped PSNR runs and print them as one JSON line")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-rows", action="store_true", help="skip the row-sampling variant's measurement")
    ap.add_argument("--converge-iters", type=int, default=60)
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other benchmark configurations (30^3, 64^5, 1024x1024x256, sampled 128^4)")
    ap.add_argument("--configs-only", action="store_true",
                    help="run only the other configurations and print them as one JSON line")
    ap.add_argument("--only-config", default=None, choices=[None, "tiny3", "cfg64", "video", "grad128"],
                    help="with --configs-only: run one configuration (short runs for profiling)")
    ap.add_argument("--conv-iters", type=int, default=None,
                    help="override the iteration limit of the configurations' time-to-1e-3 runs")
    ap.add_argument("--video-rank80", action="store_true",
                    help="run only the 1920x1080x3x50 rank [80,80,3,20] completion and print it as one JSON line")
    ap.add_argument("--no-video-rank80", action="store_true",
                    help="skip the 1920x1080x3x50 rank [80,80,3,20] completion in the full run")
    ap.add_argument("--cpu-budget", type=float, default=3.0,
                    help="seconds of oracle work per configuration and thread setting (0: skip)")
    ap.add_argument("--oracle-probe", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--oracle-budget", type=float, default=3.0, help=argparse.SUPPRESS)
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


def workload_config(w, precision):
    return {
        "workload": f"{w.name}: {'x'.join(map(str, w.dims))} TR ranks {w.ranks[0]}, "
                    f"{int(w.missing * 100)}% missing, {int(w.outlier_frac * 100)}% outliers "
                    f"U[-10 std,10 std] + N(0,{w.noise_var:g}) noise, full-tensor AWRTRD step "
                    f"(all {len(w.dims)} cores)",
        "dims": list(w.dims), "ranks": list(w.ranks), "precision": precision,
        "sigma": "adaptive (per iteration, 2^20-entry probe)",
        "l2": "inputs larger than L2 (400 MB tensor + 12.5 MB mask per pass), no flush",
        "seeds": {"data": w.data_seed, "init": w.init_seed},
    }


# ----------------------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi sampled every 200 ms during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sms, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sms.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sms) if sms else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sms)}


# ----------------------------------------------------------------------------- problem
def build_problem(w, torch, prec):
    """Seeded synthetic tensor on the device: X_true = R(Z_true) by the library's
    reconstruction kernel, then noise and outliers from the workload generator."""
    from paper_2305_09044_gb300 import TRD, synth
    truth = synth.gaussian_cores(w.dims, w.ranks, w.data_seed)
    t = TRD(w.dims, w.ranks, prec)
    Xt = t.reconstruct_from(truth)
    torch.cuda.synchronize()
    xt_host = Xt.cpu().numpy().astype(np.float64).reshape(w.dims, order="F")
    c = synth.draw_corruption(w)
    X = synth.assemble(xt_host, c, kind=w.outlier_kind).astype(np.float32).reshape(-1, order="F")
    words = synth.pack_mask(c.mask)
    del xt_host
    Xh = torch.from_numpy(X).pin_memory()
    Mh = torch.from_numpy(words.view(np.int32)).pin_memory()
    Xd = Xh.cuda()
    Md = Mh.cuda()
    t.set_data(Xd, Md)
    return t, Xt, (Xh, Mh), (Xd, Md), c


def timed_steps(t, steps, warmup, world, local, torch, kernel_launches):
    """Warm up, then time `steps` trd_step calls with CUDA events on the handle's stream;
    inside the timed region only the fused data passes are traced by the library (events
    around each launch, level 1).  A few more steps after it, traced at every phase
    (level 2), give the per-phase breakdown; they are not part of the timing."""
    # warm-up at the timed tracing level: the first steps run eagerly, the third is captured
    # as a CUDA graph, so the timed steps are graph replays
    t.set_profiling(1)
    for _ in range(max(warmup, 3)):
        t.step(sigma=-1.0)
    t.get_profile(reset=True)
    _barrier(world)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    l0 = kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(t.stream)
    for _ in range(steps):
        t.step(sigma=-1.0)
    ev1.record(t.stream)
    torch.cuda.synchronize()
    launches = kernel_launches() - l0
    ck = clocks.stop()
    prof = t.get_profile(reset=True)
    t.set_profiling(2)
    for _ in range(3):
        t.step(sigma=-1.0)
    phases = t.get_profile(reset=True)
    t.set_profiling(False)
    prof["phases_untimed"] = phases
    ms = _max_over_ranks(ev0.elapsed_time(ev1), world)
    return ms, prof, launches, ck


def recorded_traffic(prec):
    """DRAM bytes per launch of the dominant kernel from the committed ncu summary, or None
    when the kernel source changed since those counters were taken."""
    import hashlib
    import re
    name, src = {"bf16": ("k_pass_tc_100x4_rank8.md", "pass_tc.cuh"),
                 "tf32x3": ("k_pass_tc_tf32_100x4_rank8.md", "pass_tc.cuh")}.get(
        prec, ("k_pass_simt_100x4_rank8.md", "pass_simt.cu"))
    try:
        txt = open(os.path.join(ROOT, "profiles", name)).read()
        m = re.search(r"traffic_bytes_per_launch: (\d+) .*source sha1 ([0-9a-f]+)", txt)
        code = open(os.path.join(ROOT, "paper_2305_09044_gb300", "csrc", src), "rb").read()
        if m and hashlib.sha1(code).hexdigest().startswith(m.group(2)):
            return int(m.group(1))
    except OSError:
        pass
    return None


def roofline(prec, prof, w, measured=None):
    pk, src = peaks()
    Kp = w.ranks[0] * w.ranks[len(w.dims) // 2]
    n_slots = int(np.prod(w.dims))
    launches_pass = prof["pass1_n"] + prof["pass2_n"]
    pass_ms = (prof["pass1_ms"] + prof["pass2_ms"]) / max(launches_pass, 1)
    hbm_bytes = n_slots * (4 + 1 / 8)                   # x (FP32) + mask bit per slot
    line_search = None
    if prec == "bf16":
        # pass 1 (k_pass_tc) reads x and the mask bit and writes the slot's weight byte; the
        # line search (k_pass_wls) reads that byte back: one byte per slot
        launches_pass = prof["pass1_n"]
        pass_ms = prof["pass1_ms"] / max(launches_pass, 1)
        hbm_bytes = n_slots * (4 + 1 / 8 + 1)
        ls_ms = prof["pass2_ms"] / max(prof["pass2_n"], 1)
        ls_bytes = n_slots * 1.0
        line_search = {"kernel": "k_pass_wls (line search from the cached weights)", "bound": "hbm",
                       "ms_per_launch": ls_ms, "launches": prof["pass2_n"],
                       "algorithmic_bytes_per_launch": ls_bytes,
                       "achieved": ls_bytes / (ls_ms / 1e3) / 1e9 if ls_ms > 0 else None,
                       "peak": pk["hbm_gbs"], "unit": "GB/s"}
        if line_search["achieved"]:
            line_search["frac"] = line_search["achieved"] / pk["hbm_gbs"]
    if prec in ("bf16", "tf32x3"):
        achieved = hbm_bytes / (pass_ms / 1e3) / 1e9
        kname = ("k_pass_tc (fused tcgen05 data pass 1: residual, weight, gradient contraction; "
                 "weights cached as bytes)" if prec == "bf16" else
                 "k_pass_tc TF32 (fused tcgen05 data pass, 3-term TF32 products, passes 1+2)")
        roof = {"kernel": kname, "bound": "hbm",
                "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / pk["hbm_gbs"], "traffic": None,
                "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)" if src == "measured" else "fallback"}
        if prec == "tf32x3" and measured and measured.get("tf32_tflops"):
            # executed tensor work: 3 product terms of 2 K' flops in each of the two GEMMs per slot
            fl = n_slots * 3 * 4 * Kp
            roof["tensor_tflops_executed"] = fl / (pass_ms / 1e3) / 1e12
            roof["tensor_peak_tf32_measured"] = measured["tf32_tflops"]
            roof["tensor_frac_executed"] = roof["tensor_tflops_executed"] / measured["tf32_tflops"]
    else:
        algo = n_slots * 4 * Kp                         # 2 Kp recon + 2 Kp contraction per slot
        sm = pk.get("sm_max_mhz", 2070.0)
        if prec == "fp32" and measured and measured.get("fp32_simt_tflops"):
            peak = measured["fp32_simt_tflops"]
            psrc = "measured in this run: cuBLAS FP32 GEMM with TF32 off (" + measured["how"] + ")"
        elif prec == "fp32":
            peak = 152 * 128 * 2 * sm * 1e6 / 1e12
            psrc = f"derived: 152 SMs x 128 FP32 lanes x 2 flop x {sm:.0f} MHz"
        elif measured and measured.get("fp64_tflops"):
            peak, psrc = measured["fp64_tflops"], "measured in this run: cuBLAS FP64 GEMM"
        else:
            peak, psrc = 1.25, "nominal GB300 FP64 rate"
        achieved = algo / (pass_ms / 1e3) / 1e12
        roof = {"kernel": "k_pass_simt (fused data pass, CUDA cores)", "bound": "alu",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "peak_source": psrc}
    roof["traffic"] = recorded_traffic(prec) if w.name == WORKLOAD else None
    roof["ms_per_launch"] = pass_ms
    roof["launches"] = launches_pass
    ph = prof.get("phases_untimed", {})
    steps = max(ph.get("stop_n", 0), 1)
    # per-phase breakdown from the untimed steps traced at every phase (event overhead
    # included there, so the phases add up to a little more than ms_per_step)
    roof["phase_ms_per_step_untimed"] = {k[:-3]: round(v / steps, 4) for k, v in ph.items()
                                         if k.endswith("_ms") and v > 0}
    roof["algorithmic_bytes_per_launch"] = hbm_bytes
    roof["hbm_gbs_achieved"] = hbm_bytes / (pass_ms / 1e3) / 1e9
    if line_search:
        roof["line_search_pass"] = line_search
    return roof


def run_ours(args, rank, world, local):
    import torch
    from paper_2305_09044_gb300 import TRD, synth
    from paper_2305_09044_gb300.binding import kernel_launches
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(local)
    precs = [args.precision] if args.precision else ["bf16", "tf32x3", "fp32"]
    measured = measure_peaks(torch) if rank == 0 else None
    w = replica_workload(synth.WORKLOADS[WORKLOAD], rank, world)
    t, Xt, host, dev, corr = build_problem(w, torch, precs[0])
    slots_per_step = len(w.dims) * int(np.prod(w.dims))

    # headline path
    t.init_cores(w.init_seed)
    ms, prof, launches, ck = timed_steps(t, args.steps, args.warmup, world, local, torch, kernel_launches)
    ms_step = ms / args.steps
    value = job_throughput(world, slots_per_step, args.steps, ms)
    prec = precs[0]

    # e2e through the public API with host buffers.  Every step's X and mask are copied from
    # pinned host memory into one of two device buffer pairs on a copy stream while the
    # previous step computes (double buffering); the step attaches its pair (trd_set_data,
    # which drops everything derived from the old contents, so the mask re-layout and the
    # probe values are recomputed every step and the steps run eagerly, without graph
    # replay), runs, and reads its report back (inside trd_step).
    Xh, Mh = host
    Xd, Md = dev
    pairs = [(Xd, Md), (torch.empty_like(Xd), torch.empty_like(Md))]
    h2d = Xh.numel() * 4 + Mh.numel() * 4
    d2h = 32 * 8
    copy_stream = torch.cuda.Stream()
    main_stream = torch.cuda.current_stream()
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    released = [torch.cuda.Event(), torch.cuda.Event()]

    def upload(j):
        copy_stream.wait_event(released[j])
        with torch.cuda.stream(copy_stream):
            pairs[j][0].copy_(Xh, non_blocking=True)
            pairs[j][1].copy_(Mh, non_blocking=True)
            copied[j].record(copy_stream)

    def e2e_steps(n):
        for j in range(2):
            released[j].record(main_stream)
        upload(0)
        for i in range(n):
            j = i % 2
            main_stream.wait_event(copied[j])
            t.set_data(*pairs[j])
            if i + 1 < n:
                upload(1 - j)
            t.step(sigma=-1.0)
            released[j].record(main_stream)

    e2e_steps(3)                # warm-up: same calls as the timed steps
    torch.cuda.synchronize()
    _barrier(world)
    t0 = time.perf_counter()
    e2e_steps(args.steps)
    torch.cuda.synchronize()
    e2e_s = _max_over_ranks((time.perf_counter() - t0) * 1e3, world) / 1e3
    e2e = {"value": job_throughput(world, slots_per_step, args.steps, e2e_s * 1e3), "unit": UNIT,
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
           "ms_per_step": e2e_s * 1e3 / args.steps,
           "note": "per step: H2D of X and mask from pinned memory (double-buffered, overlapping the "
                   "previous step), trd_set_data, trd_step with its report read back"}
    t.set_data(Xd, Md)

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": max(args.warmup, 3), "ms_per_step": ms_step, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": {"fp32": "f32", "bf16": "bf16", "fp64": "f64", "tf32x3": "tf32x3"}[prec],
           "data": "synthetic", "config": workload_config(w, prec), "iters_per_s": 1e3 / ms_step,
           "roofline": roofline(prec, prof, w, measured), "e2e": e2e, "gpu_launches": launches, "clocks": ck}
    if measured:
        out["peaks_measured_here"] = measured
    if rank == 0 and not args.no_converge:
        out["time_to_rel_err_1e-3"] = converge(t, Xt, w, args.converge_iters, torch)
    if not args.no_rows:
        out["row_sampling"] = row_sampling(t, w, torch)
    if rank == 0 and not args.no_image:
        out["image"] = [image_quality(name, prec, torch) for name in ("image", "imagec")]
        if not args.no_video_rank80:
            try:
                out["video_rank80"] = video_rank80(torch, prec)
            except Exception as exc:          # reported, so that the other legs still print
                out["video_rank80"] = {"error": f"{type(exc).__name__}: {exc}"}

    # comparison path on the same device data (FP32 CUDA-core passes)
    for other in precs[1:]:
        t2 = TRD(w.dims, w.ranks, other)
        t2.set_data(Xd, Md)
        t2.init_cores(w.init_seed)
        steps2 = max(3, args.steps // 4)
        ms2, prof2, launches2, ck2 = timed_steps(t2, steps2, 3, world, local, torch, kernel_launches)
        cmp_ = {"value": job_throughput(world, slots_per_step, steps2, ms2), "unit": UNIT, "steps": steps2,
                "ms_per_step": ms2 / steps2, "iters_per_s": 1e3 * steps2 / ms2,
                "roofline": roofline(other, prof2, w, measured), "gpu_launches": launches2, "clocks": ck2}
        if rank == 0 and not args.no_converge:
            cmp_["time_to_rel_err_1e-3"] = converge(t2, Xt, w, args.converge_iters, torch)
        out[other] = cmp_
        t2.close()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(w, corr, budget_s=15.0)
        if args.cpu_budget > 0:
            out["cpu_baseline"]["threads"] = {"one_thread": oracle_probe("subtensor", WORKLOAD, 1, args.cpu_budget),
                                              "all_cores": oracle_probe("subtensor", WORKLOAD, os.cpu_count() or 1,
                                                                        args.cpu_budget)}
    t.close()
    del host, dev, Xt
    torch.cuda.empty_cache()
    if rank == 0 and not args.no_configs:
        out["configs"] = other_configs(args, torch, measured)
    if rank == 0:
        print(json.dumps(out), flush=True)


def other_configs(args, torch, measured):
    """The other benchmark configurations on this GPU (each with its own roofline and CPU
    baseline): 30^3 FP64 trajectory, 64^5 and 1024 x 1024 x 256 RStS iterations, sampled
    128^4 forward + backward."""
    pk, _ = peaks()
    if measured:
        _MEASURED.update(measured)
    budget = 0.0 if args.no_cpu_baseline else args.cpu_budget
    want = [args.only_config] if args.only_config else ["tiny3", "cfg64", "video", "grad128"]
    ci = args.conv_iters
    res = {}
    if "tiny3" in want:
        res["tiny3"] = run_tiny(torch, pk, budget)
    if "cfg64" in want:
        # from the random initialisation the 64^5 rank-10 problem sits near relative error 1 for
        # tens of iterations before it converges (the oracle shows the same plateau on small
        # analogues), so its time to 1e-3 gets a longer iteration limit
        res["cfg64"] = run_sketched(torch, pk, "cfg64", ["bf16"], 10, budget,
                                    conv_iters=400 if ci is None else ci, conv_budget=4.0)
    if "video" in want:
        res["video"] = run_sketched(torch, pk, "video", ["bf16", "fp32"], 10, budget,
                                    conv_iters=60 if ci is None else ci, conv_budget=6.0)
    if "grad128" in want:
        res["grad128"] = run_sampled(torch, pk, 5, budget)
    return res


def row_sampling(t, w, torch, J=1 << 16, updates=8):
    """The uniform-row-sampling variant (the paper's ablation): per core update, J rows of the
    subchain unfolding drawn i.i.d. uniformly (numpy, seeded), the fibres gathered, then the
    residual / gradient / scaled-step / line-search path on them.  Device time of the whole
    update (gather included) with CUDA events; the host draw and index upload are outside."""
    rng = np.random.default_rng(w.sample_seed + 17)
    N = len(w.dims)
    stream = t.stream
    total, slots = 0.0, 0
    for q in range(updates + 2):
        k = q % N
        rows = np.stack([rng.integers(0, w.dims[m], J) if m != k else np.zeros(J, dtype=np.int64)
                         for m in range(N)], axis=1)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        t.sample_rows(k, rows)
        t.residual_weights(k, 2.0)
        t.core_gradient(k)
        t.core_update(k, -1e-10)
        b.record(stream)
        torch.cuda.synchronize()
        if q >= 2:                       # two warm-up updates
            total += a.elapsed_time(b)
            slots += w.dims[k] * J
    t.sample_subtensor(0, None)
    return {"value": slots / (total / 1e3), "unit": UNIT, "rows_per_update": J, "updates": updates,
            "ms_per_update": total / updates, "note": "one core update per timed interval (sample gather, "
            "both data passes, gradient, FGMC Gram, LDL^T solve, line search); sigma fixed at 2"}


def image_quality(name, prec, torch, max_iters=30, tol=1e-3):
    """Sec. 5's image experiments on a seeded image-shaped tensor: AWRTRD with the adaptive
    width for at most 30 iterations or until e < 1e-3 (the paper's limits); PSNR against
    the clean tensor (peak = its range, i.e. data on the [0, 1] scale) before, during and
    after, evaluated outside the timed steps."""
    from paper_2305_09044_gb300 import synth
    w = synth.WORKLOADS[name]
    t, Xt, host, dev, corr = build_problem(w, torch, prec)
    xt = Xt.cpu().numpy()
    peak = float(xt.max() - xt.min())
    X = host[0].numpy()
    obs = corr.mask.reshape(-1, order="F")
    noisy = 10 * math.log10(peak ** 2 / float(np.mean((X[obs].astype(np.float64) - xt[obs]) ** 2)))
    del xt, X
    t.init_cores(w.init_seed)
    trace = [t.psnr(Xt, peak)]
    stream = t.stream
    total, it, e = 0.0, 0, math.inf
    while it < max_iters and e >= tol:
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r = t.step(sigma=-1.0)
        b.record(stream)
        torch.cuda.synchronize()
        total += a.elapsed_time(b)
        e = r["e"]
        it += 1
        trace.append(t.psnr(Xt, peak))
    # two more steps traced at every phase, after the measured run (not part of it)
    t.set_profiling(2)
    t.get_profile(reset=True)
    for _ in range(2):
        t.step(sigma=-1.0)
    ph = t.get_profile(reset=True)
    t.set_profiling(False)
    t.close()
    return {"phase_ms_per_step_untimed": {k[:-3]: round(v / 2, 4) for k, v in ph.items()
                                          if k.endswith("_ms") and v > 0},
            "workload": w.name, "dims": list(w.dims), "ranks": list(w.ranks), "missing": w.missing,
            "noise": "0.8 N(0, 1e-3) + 0.2 N(0, 0.5) on the [0, 1] scale", "precision": prec,
            "psnr_noisy_observed_db": noisy, "psnr_init_db": trace[0], "psnr_db": trace[-1],
            "iters": it, "e": e, "seconds": total / 1e3,
            "psnr_trace_db": [round(p, 2) for p in trace]}


def video_rank80(torch, prec, max_iters=6, budget_s=60.0):
    """Sec. 5's video completion setting on a seeded video-shaped tensor: 1920 x 1080 x 3 x 50
    at the paper's TR rank [80, 80, 3, 20] (K = 6400 for the first core), 70 % missing,
    mixture noise, SAWRTRD with RStS (J = 3e4 sampled fibres when a frame mode is updated) and
    the adaptive width.  Device time per iteration and PSNR against the clean tensor, evaluated
    outside the timed steps; at most max_iters iterations or budget_s seconds of steps."""
    from paper_2305_09044_gb300 import synth
    w = synth.WORKLOADS["videop"]
    N = len(w.dims)
    t, Xt, X, M = device_problem(w, torch, prec)
    peak = float(Xt.max() - Xt.min())
    noisy = 10 * math.log10(peak ** 2 / float(((X.double() - Xt.double()) ** 2).mean()))
    del X
    kw = {"sketch": [w.sketch] * N, "sigma": -1.0, "seed": w.sample_seed}
    slots = [int(np.prod([w.dims[m] if m == k else min(w.sketch, w.dims[m]) for m in range(N)]))
             for k in range(N)]
    t.init_cores(w.init_seed)
    trace = [t.psnr(Xt, peak)]
    stream = t.stream
    times = []
    e = math.inf
    while len(times) < max_iters and sum(times) < budget_s * 1e3:
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r = t.step(**kw)
        b.record(stream)
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
        e = r["e"]
        trace.append(t.psnr(Xt, peak))
    t.set_profiling(2)
    t.get_profile(reset=True)
    t.step(**kw)
    ph = t.get_profile(reset=True)
    t.set_profiling(False)
    t.close()
    del Xt, M
    torch.cuda.empty_cache()
    return {"workload": f"{w.name}: {'x'.join(map(str, w.dims))} TR rank {list(w.ranks)}, "
                        f"{int(w.missing * 100)}% missing, mixture noise 0.8 N(0, 1e-3) + 0.2 N(0, 0.5) "
                        f"on the [0, 1] scale on every entry, RStS sketch {w.sketch} per non-updated mode, "
                        f"adaptive sigma",
            "precision": prec, "K_per_core": [w.ranks[k] * w.ranks[(k + 1) % N] for k in range(N)],
            "sampled_slots_per_core": slots, "iters": len(times),
            "ms_per_iter": [round(x, 2) for x in times], "ms_per_iter_after_first": (
                float(np.mean(times[1:])) if len(times) > 1 else None),
            "e": e, "psnr_noisy_all_entries_db": noisy, "psnr_init_db": trace[0], "psnr_db": trace[-1],
            "psnr_trace_db": [round(p, 2) for p in trace],
            "phase_ms_one_iteration_untimed": {k[:-3]: round(v, 2) for k, v in ph.items()
                                              if k.endswith("_ms") and v > 0},
            "data": "synthetic; corruption drawn on the device by torch's seeded generator"}


def converge(t, Xt, w, iters, torch):
    """Iterations and device time from a fresh initialisation until the recovery error
    ||R(Z) - X_true|| / ||X_true|| <= 1e-3 (error evaluated outside the timed steps)."""
    t.init_cores(w.init_seed)
    stream = t.stream
    total = 0.0
    err = t.recovery_error(Xt)
    for it in range(iters):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        t.step(sigma=-1.0)
        b.record(stream)
        torch.cuda.synchronize()
        total += a.elapsed_time(b)
        err = t.recovery_error(Xt)
        if err <= 1e-3:
            return {"reached": True, "iters": it + 1, "seconds": total / 1e3, "rel_err": err}
    return {"reached": False, "iters": iters, "seconds": total / 1e3, "rel_err": err}


# ----------------------------------------------------------------------------- other configurations
def measure_peaks(torch):
    """Denominators that MEASURED_PEAKS.json does not hold, measured here the same way (a
    library GEMM, best of five CUDA-event timed runs after two warm-ups): FP64, FP32 on the CUDA
    cores (TF32 off) and TF32.  Only the denominators come from library code."""
    out = {}
    prev = torch.backends.cuda.matmul.allow_tf32
    try:
        for name, dtype, n, tf32 in (("fp64_tflops", torch.float64, 4096, False),
                                     ("fp32_simt_tflops", torch.float32, 8192, False),
                                     ("tf32_tflops", torch.float32, 8192, True)):
            torch.backends.cuda.matmul.allow_tf32 = tf32
            a = torch.randn(n, n, device="cuda", dtype=dtype)
            b = torch.randn(n, n, device="cuda", dtype=dtype)
            for _ in range(2):
                torch.matmul(a, b)
            best = math.inf
            for _ in range(5):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b)
                e1.record()
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1) / 1e3)
            out[name] = 2.0 * n ** 3 / best / 1e12
            del a, b
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    out["how"] = ("torch.matmul (cuBLAS) n^3 GEMM, 2 n^3 flops, best of 5: FP64 n = 4096, FP32 with TF32 "
                  "off and TF32 n = 8192; on this run's GPU")
    return out


def device_problem(w, torch, prec, chunk=1 << 26):
    """Seeded synthetic tensor built on the device, for the ~1e9-entry workloads: X_true =
    R(Z_true) by the library's reconstruction kernel (cores from the workload generator), then
    the workload's corruption drawn chunk by chunk by torch's seeded device generator (same
    distributions as the host recipe: Bernoulli mask, outliers U[-10 std, 10 std] on observed
    entries or salt-and-pepper at the clean tensor's max / min, additive Gaussian noise, or the
    two-component mixture noise on every entry), and the mask bit-packed on the device."""
    from paper_2305_09044_gb300 import TRD, synth
    truth = synth.gaussian_cores(w.dims, w.ranks, w.data_seed, w.smooth_modes, w.smooth_width)
    t = TRD(w.dims, w.ranks, prec)
    Xt = t.reconstruct_from(truth)
    n = Xt.numel()
    g = torch.Generator(device="cuda")
    g.manual_seed(w.data_seed)
    std = float(Xt.std())
    lo, hi = float(Xt.min()), float(Xt.max())
    X = torch.empty_like(Xt)
    words = ((n + 31) // 32 + 3) // 4 * 4
    M = torch.zeros(words, dtype=torch.int32, device="cuda")
    shifts = torch.arange(32, device="cuda", dtype=torch.int64)
    for s in range(0, n, chunk):
        c = min(chunk, n - s)
        m = torch.rand(c, generator=g, device="cuda") < (1.0 - w.missing)
        out = torch.rand(c, generator=g, device="cuda") < w.outlier_frac
        u = torch.rand(c, generator=g, device="cuda") * 2.0 - 1.0
        x = Xt[s:s + c]
        if w.noise_var > 0:
            x = x + math.sqrt(w.noise_var) * torch.randn(c, generator=g, device="cuda")
        if w.outlier_kind == "saltpepper":
            x = torch.where(out, torch.where(u > 0, torch.full_like(x, hi), torch.full_like(x, lo)), x)
        elif w.outlier_kind == "gmm":
            sd = torch.where(out, math.sqrt(synth.GMM_VARS[1]), math.sqrt(synth.GMM_VARS[0]))
            x = x + (hi - lo) * sd * torch.randn(c, generator=g, device="cuda")
            del sd
        else:
            x = torch.where(out & m, 10.0 * std * u, x)
        X[s:s + c] = x
        pad = (-c) % 32
        mb = torch.nn.functional.pad(m, (0, pad)).view(-1, 32).to(torch.int64)
        packed = ((mb << shifts).sum(dim=1) & 0xFFFFFFFF)
        packed = torch.where(packed >= 2 ** 31, packed - 2 ** 32, packed).to(torch.int32)
        M[s // 32: s // 32 + packed.numel()] = packed
        del m, out, u, x, mb, packed
    t.set_data(X, M)
    return t, Xt, X, M


def oracle_probe(kind, name, threads, budget_s):
    """Time the FP64 oracle on a bounded sample of workload `name` in a child process limited
    to `threads` BLAS/OpenMP threads (the thread count of numpy's BLAS is fixed at its import).
    Returns the child's JSON result."""
    env = dict(os.environ)
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[var] = str(threads)
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-probe", f"{kind}:{name}",
                        "--oracle-budget", str(budget_s)], env=env, capture_output=True, text=True,
                       timeout=600)
    for line in r.stdout.splitlines()[::-1]:
        if line.startswith("{"):
            res = json.loads(line)
            res["threads"] = threads
            return res
    return {"error": (r.stderr or r.stdout)[-300:], "threads": threads}


def oracle_probe_main(spec, budget_s):
    """Child side of oracle_probe: one bounded sample of the named workload."""
    from oracle import trd_oracle as O
    from paper_2305_09044_gb300 import synth
    kind, name = spec.split(":")
    w = synth.WORKLOADS[name]
    t0 = time.perf_counter()
    if kind == "trajectory":
        # the 30^3 workload: full oracle iterations (Algorithm 1) with the adaptive width
        truth = synth.gaussian_cores(w.dims, w.ranks, w.data_seed)
        Xt = O.reconstruct_unfold(truth)
        c = synth.draw_corruption(w)
        X = synth.assemble(Xt, c).astype(np.float32).astype(np.float64)
        P = c.mask.astype(np.float64)
        cores = O.init_cores(w.dims, w.ranks, seed=w.init_seed)
        obs = P > 0
        rms = float(np.sqrt(np.mean(X[obs] ** 2)))
        D, sigma, its = O.D_matrix(cores), None, 0
        t0 = time.perf_counter()
        while its < 100 and (its == 0 or time.perf_counter() - t0 < budget_s):
            sigma = O.adaptive_sigma((X - O.reconstruct(cores))[obs], rms, sigma)
            cores, e, D, steps = O.sawrtrd_iteration(X, P, cores, sigma, its, D_prev=D)
            its += 1
        dt = time.perf_counter() - t0
        print(json.dumps({"unit": "iterations/s", "value": its / dt, "iters": its, "seconds": dt,
                          "sample": f"{its} oracle iterations of Algorithm 1 on the full 30^3 workload"}))
        return
    if kind == "sketch":
        # one RStS core update per sample on a synthetic tensor of the workload's sketch shape
        # (the gathered sketch itself: dims I_k x s^(N-1)), repeated within the budget
        N = len(w.dims)
        rng = np.random.default_rng(w.data_seed)
        k = 1
        sdims = [w.dims[m] if m == k else min(w.sketch, w.dims[m]) for m in range(N)]
        cores = O.init_cores(sdims, w.ranks, seed=w.init_seed)
        X = O.reconstruct_unfold([c * 1.01 for c in cores]) + 0.01 * rng.standard_normal(sdims)
        P = (rng.random(sdims) < 1.0 - w.missing).astype(np.float64)
        slots = int(np.prod(sdims))
        done = 0
        t0 = time.perf_counter()
        while done == 0 or time.perf_counter() - t0 < budget_s:
            O.core_update(X, P, cores, k, 2.0)
            done += 1
        dt = time.perf_counter() - t0
        print(json.dumps({"unit": UNIT, "value": done * slots / dt, "updates": done, "seconds": dt,
                          "sample": f"{done} oracle core updates (k = {k + 1}) on a {'x'.join(map(str, sdims))} "
                                    f"sketch-shaped tensor (TR ranks {w.ranks[0]})"}))
        return
    if kind == "sampled":
        # the sampled loss and its gradient at a subset of the workload's entries
        Msub = 1 << 14
        cores = O.init_cores(w.dims, w.ranks, seed=w.init_seed)
        rng = np.random.default_rng(w.sample_seed)
        idx = np.stack([rng.integers(0, d, Msub) for d in w.dims], axis=1)
        x = rng.standard_normal(Msub)
        done = 0
        t0 = time.perf_counter()
        while done == 0 or time.perf_counter() - t0 < budget_s:
            O.sampled_loss_grad_vec(cores, idx, x, 1.0)
            done += 1
        dt = time.perf_counter() - t0
        print(json.dumps({"unit": "sampled entries/s (fwd+bwd)", "value": done * Msub / dt, "evals": done,
                          "seconds": dt, "sample": f"{done} oracle loss+gradient evaluations at {Msub} sampled "
                                                    f"entries of the {'x'.join(map(str, w.dims))} rank-{w.ranks[0]} model"}))
        return
    if kind == "subtensor":
        X, P, cores, sigma, sub = oracle_sample(w, None)
        slots = int(np.prod(sub))
        done, k = 0, 0
        t0 = time.perf_counter()
        while done == 0 or time.perf_counter() - t0 < budget_s:
            cores = O.core_update(X, P, cores, k % len(sub), sigma).cores
            done += 1
            k += 1
        dt = time.perf_counter() - t0
        print(json.dumps({"unit": UNIT, "value": done * slots / dt, "updates": done, "seconds": dt,
                          "sample": f"{done} oracle core updates on the {'x'.join(map(str, sub))} sub-tensor"}))
        return
    raise ValueError(kind)


def cpu_pair(kind, name, budget_s):
    """The oracle at 1 thread and at every host core."""
    ncores = os.cpu_count() or 1
    one = oracle_probe(kind, name, 1, budget_s)
    allc = oracle_probe(kind, name, ncores, budget_s)
    return {"kind": "oracle", "cores": ncores, "one_thread": one, "all_cores": allc}


def timed_device_steps(t, steps, warmup, torch, step_kw):
    """CUDA-event time of `steps` trd_step calls after `warmup` (tracing off), then a few
    untimed steps traced at every phase for the breakdown; returns ms per step and phases."""
    from paper_2305_09044_gb300.binding import kernel_launches
    for _ in range(warmup):
        t.step(**step_kw)
    torch.cuda.synchronize()
    l0 = kernel_launches()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(t.stream)
    for _ in range(steps):
        t.step(**step_kw)
    b.record(t.stream)
    torch.cuda.synchronize()
    launches = (kernel_launches() - l0) / steps
    ms = a.elapsed_time(b) / steps
    t.set_profiling(2)
    t.get_profile(reset=True)
    for _ in range(2):
        t.step(**step_kw)
    ph = t.get_profile(reset=True)
    t.set_profiling(False)
    return ms, ph, launches


def converge_steps(t, Xt, step_kw, max_iters, budget_s, torch):
    """Device time from a fresh initialisation until ||R(Z) - X_true|| / ||X_true|| <= 1e-3
    (evaluated outside the timed steps), at most max_iters iterations or budget_s of device time."""
    stream = t.stream
    total, err, it = 0.0, t.recovery_error(Xt), 0
    while it < max_iters and total < budget_s * 1e3:
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        t.step(**step_kw)
        b.record(stream)
        torch.cuda.synchronize()
        total += a.elapsed_time(b)
        it += 1
        err = t.recovery_error(Xt)
        if err <= 1e-3:
            return {"reached": True, "iters": it, "seconds": total / 1e3, "rel_err": err}
    return {"reached": False, "iters": it, "seconds": total / 1e3, "rel_err": err}


def phase_summary(ph, steps=2):
    return {k[:-3]: round(v / steps, 4) for k, v in ph.items() if k.endswith("_ms") and v > 0}


def pass_roofline(ph, slots_per_pass, pk, label, steps=2, Kp=None, tf32_peak=None, cached_weights=False):
    """Fused data passes of the traced steps: algorithmic bytes (x and the mask bit per slot)
    over the average pass time, against the measured HBM copy bandwidth; for the TF32 passes
    also the executed tensor flops (3 product terms) against the measured TF32 peak.  With
    cached_weights (BF16), pass 1 also writes a weight byte per slot and the line-search pass,
    reported on its own, reads it back."""
    n = ph.get("pass1_n", 0) + ph.get("pass2_n", 0)
    if n == 0:
        return None
    ms = (ph["pass1_ms"] + ph["pass2_ms"]) / n
    byt = slots_per_pass * (4 + 1 / 8)
    if cached_weights and ph.get("pass1_n", 0):
        n = ph["pass1_n"]
        ms = ph["pass1_ms"] / n
        byt = slots_per_pass * (4 + 1 / 8 + 1)
    gbs = byt / (ms / 1e3) / 1e9
    r = {"kernel": label, "bound": "hbm", "achieved": gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
         "frac": gbs / pk["hbm_gbs"], "ms_per_launch": ms, "launches": n, "algorithmic_bytes_per_launch": byt}
    if cached_weights and ph.get("pass2_n", 0):
        ls = ph["pass2_ms"] / ph["pass2_n"]
        lb = slots_per_pass * 1.0
        r["line_search_pass"] = {"kernel": "k_pass_wls", "ms_per_launch": ls, "launches": ph["pass2_n"],
                                 "algorithmic_bytes_per_launch": lb, "achieved": lb / (ls / 1e3) / 1e9,
                                 "frac": lb / (ls / 1e3) / 1e9 / pk["hbm_gbs"], "unit": "GB/s"}
    if Kp and tf32_peak:
        fl = slots_per_pass * 3 * 4 * Kp
        r["tensor_tflops_executed"] = fl / (ms / 1e3) / 1e12
        r["tensor_frac_of_tf32"] = r["tensor_tflops_executed"] / tf32_peak
    return r


_MEASURED = {}


def measured_fp64(pk):
    return _MEASURED.get("fp64_tflops") or 1.25


def fp64_roofline(w, ph, fp64_peak, steps=2):
    """FP64 factorisation and solves of the scaled step (Eq. sg / Eq. hI) per iteration, from
    the traced phases: K^3 / 3 flops per Cholesky (K = r_k r_{k+1}), 2 I_k K^2 per pair of
    substitutions, against the FP64 GEMM peak measured in this run.  Latency-bound at these
    sizes (K <= 400); reported so the fraction is on record."""
    N = len(w.dims)
    Ks = [w.ranks[k] * w.ranks[(k + 1) % N] for k in range(N)]
    chol = sum(K ** 3 / 3.0 for K in Ks)
    solve = sum(2.0 * w.dims[k] * Ks[k] ** 2 for k in range(N))
    c_ms = ph.get("cholesky_ms", 0.0) / steps
    s_ms = ph.get("solve_ms", 0.0) / steps
    r = {"K": Ks, "peak_fp64_tflops": fp64_peak, "peak_source": "measured in this run (cuBLAS FP64 GEMM)"}
    if c_ms > 0:
        r["cholesky_ms_per_iter"] = c_ms
        r["cholesky_tflops"] = chol / (c_ms / 1e3) / 1e12
        r["cholesky_frac"] = r["cholesky_tflops"] / fp64_peak
    if s_ms > 0:
        r["solve_ms_per_iter"] = s_ms
        r["solve_tflops"] = solve / (s_ms / 1e3) / 1e12
        r["solve_frac"] = r["solve_tflops"] / fp64_peak
    return r


def run_tiny(torch, pk, budget):
    """Benchmark configuration 1: 30^3 rank 3, 30 % missing, 10 % outliers, adaptive width,
    100 iterations on the FP64 path (launch-latency bound)."""
    from paper_2305_09044_gb300 import TRD, synth
    w = synth.WORKLOADS["tiny3"]
    t, Xt, host, dev, corr = build_problem(w, torch, "fp64")
    t.init_cores(w.init_seed)
    kw = {"sigma": -1.0}
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(t.stream)
    for _ in range(100):
        t.step(**kw)
    b.record(t.stream)
    torch.cuda.synchronize()
    ms100 = a.elapsed_time(b)
    err = t.recovery_error(Xt)
    ms, ph, launches = timed_device_steps(t, 20, 3, torch, kw)
    t.close()
    slots = 3 * 27000
    res = {"workload": "tiny3: 30^3 TR ranks 3, 30% missing, 10% outliers, adaptive sigma, FP64, 100 iterations",
           "precision": "fp64", "seconds_100_iters": ms100 / 1e3, "iters_per_s": 100 / (ms100 / 1e3),
           "ms_per_iter_steady": ms, "sampled_entries_per_s": slots / (ms / 1e3),
           "kernel_launches_per_iter": launches, "rel_err_after_100": err,
           "roofline": {"bound": "latency", "note": "27,000-slot passes: every kernel is a few microseconds; the "
                        "iteration is bound by the chain of dependent launches (replayed as one CUDA graph)",
                        "us_per_launch": ms * 1e3 / max(launches, 1)},
           "phase_ms_per_step_untimed": phase_summary(ph)}
    if budget:
        res["cpu_baseline"] = cpu_pair("trajectory", "tiny3", budget)
    return res


def run_sketched(torch, pk, name, precs, steps, budget, conv_iters, conv_budget):
    """Benchmark configurations 3 (64^5 rank 10, sketch 24 per non-updated mode) and 4
    (1024 x 1024 x 256 rank 16, sketch 128 x 128 x full): SAWRTRD iterations with the RStS
    gather inside every core update; iterations/s, sampled entries/s, per-phase times, the
    gather's and the data passes' rooflines, and time to recovery error 1e-3 per precision."""
    from paper_2305_09044_gb300 import synth
    w = synth.WORKLOADS[name]
    N = len(w.dims)
    slots = [int(np.prod([w.dims[m] if m == k else min(w.sketch, w.dims[m]) for m in range(N)]))
             for k in range(N)]
    kw = {"sketch": [w.sketch] * N, "sigma": -1.0, "seed": w.sample_seed}
    out = {"workload": f"{w.name}: {'x'.join(map(str, w.dims))} TR ranks {w.ranks[0]}, "
                       f"{int(w.missing * 100)}% missing, {int(w.outlier_frac * 100)}% "
                       f"{'salt-and-pepper' if w.outlier_kind == 'saltpepper' else 'outliers U[-10 std,10 std]'}, "
                       f"RStS sketch {w.sketch} per non-updated mode, adaptive sigma",
           "slots_per_iteration": sum(slots),
           "data": "synthetic; corruption drawn on the device by torch's seeded generator"}
    t, Xt, X, M = device_problem(w, torch, precs[0])
    for prec in precs:
        if prec != precs[0]:
            t.close()
            from paper_2305_09044_gb300 import TRD
            t = TRD(w.dims, w.ranks, prec)
            t.set_data(X, M)
        t.init_cores(w.init_seed)
        ms, ph, launches = timed_device_steps(t, steps, 3, torch, kw)
        # average per core update of the traced steps
        gather_ms = ph.get("gather_ms", 0.0) / max(ph.get("gather_n", 1), 1)
        gbytes = np.mean(slots) * (4 + 1 / 8) * 2          # read x + bit, write x_I + bit
        leg = {"ms_per_iter": ms, "iters_per_s": 1e3 / ms, "sampled_entries_per_s": sum(slots) / (ms / 1e3),
               "kernel_launches_per_iter": launches, "phase_ms_per_step_untimed": phase_summary(ph)}
        leg["roofline_pass"] = pass_roofline(ph, np.mean(slots), pk,
                                             f"fused data pass ({prec})", Kp=None,
                                             cached_weights=(prec == "bf16"))
        if gather_ms > 0:
            leg["roofline_gather"] = {"kernel": "k_gather (RStS sketch X_I, P_I)", "bound": "hbm",
                                      "achieved": gbytes / (gather_ms / 1e3) / 1e9, "peak": pk["hbm_gbs"],
                                      "unit": "GB/s", "frac": gbytes / (gather_ms / 1e3) / 1e9 / pk["hbm_gbs"],
                                      "ms_per_launch": gather_ms,
                                      "algorithmic_bytes_per_launch": gbytes}
        leg["fp64_kernels"] = fp64_roofline(w, ph, measured_fp64(pk))
        t.init_cores(w.init_seed)
        leg["time_to_rel_err_1e-3"] = converge_steps(t, Xt, kw, conv_iters, conv_budget, torch)
        out[prec] = leg
    t.close()
    del Xt, X, M
    torch.cuda.empty_cache()
    if budget:
        out["cpu_baseline"] = cpu_pair("sketch", name, budget)
    return out


def run_sampled(torch, pk, steps, budget):
    """Benchmark configuration 5: sampled correntropy loss of a 128^4 rank-20 TR model at
    2^24 observed entries (10 % outliers), forward + hand-written adjoint through the C ABI,
    FP32; forward+backward evaluations per second and sampled entries per second."""
    from paper_2305_09044_gb300 import TRD, synth
    w = synth.WORKLOADS["grad128"]
    t = TRD(w.dims, w.ranks, "fp32")
    n = int(np.prod(w.dims))
    g = torch.Generator(device="cuda")
    g.manual_seed(w.sample_seed)
    lin = torch.randperm(n, generator=g, device="cuda")[: w.n_sampled].sort().values
    idx = torch.empty((lin.numel(), 4), dtype=torch.int32, device="cuda")
    rem = lin.clone()
    for m, d in enumerate(w.dims):
        idx[:, m] = (rem % d).to(torch.int32)
        rem //= d
    del rem, lin

    def abi(cs):
        return [torch.from_numpy(np.ascontiguousarray(Z.transpose(1, 2, 0))).float().cuda() for Z in cs]

    # the clean model at the sampled entries (x_hat = -residual against x = 0), then 10 % of the
    # entries replaced by outliers U[-10 std, 10 std] (seeded device generator)
    truth = abi(synth.gaussian_cores(w.dims, w.ranks, w.data_seed))
    xh = torch.empty(idx.shape[0], dtype=torch.float32, device="cuda")
    t.sampled_fwd(truth, idx, torch.zeros_like(xh), 1.0, resid=xh)
    xh.neg_()
    gd = torch.Generator(device="cuda")
    gd.manual_seed(w.data_seed)
    out = torch.rand(xh.numel(), generator=gd, device="cuda") < w.outlier_frac
    u = torch.rand(xh.numel(), generator=gd, device="cuda") * 2.0 - 1.0
    x = torch.where(out, 10.0 * float(xh.std()) * u, xh).contiguous()
    del truth, xh, out, u
    cores = abi(synth.gaussian_cores(w.dims, w.ranks, w.init_seed))
    sigma = 1.0
    grads = [torch.empty_like(c) for c in cores]
    for _ in range(3):
        t.sampled_fwd(cores, idx, x, sigma)
        t.sampled_bwd(cores, idx, x, sigma, 1.0, grads)
    torch.cuda.synchronize()
    a, b, c2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    fwd_ms = bwd_ms = 0.0
    for _ in range(steps):
        a.record(t.stream)
        t.sampled_fwd(cores, idx, x, sigma)
        b.record(t.stream)
        t.sampled_bwd(cores, idx, x, sigma, 1.0, grads)
        c2.record(t.stream)
        torch.cuda.synchronize()
        fwd_ms += a.elapsed_time(b)
        bwd_ms += b.elapsed_time(c2)
    fwd_ms /= steps
    bwd_ms /= steps
    Mn = int(idx.shape[0])
    K = w.ranks[0] * w.ranks[2]
    # per entry: index (16 B) + value (4 B) from HBM; the merged halves (2 x 16,384 x 400 floats
    # = 52 MB) are L2-resident: the forward reads one K-float row of S_C per entry (the S_A row
    # once per group of entries), the adjoint one row of each half per entry
    hbm = Mn * 20
    l2 = Mn * K * 4
    res = {"workload": "grad128: 128^4 TR ranks 20, 10% outliers, 2^24 sampled entries, FP32 (values at the "
                       "sampled entries only)",
           "entries": Mn, "fwd_ms": fwd_ms, "bwd_ms": bwd_ms,
           "fwd_bwd_per_s": 1e3 / (fwd_ms + bwd_ms), "sampled_entries_per_s": Mn / ((fwd_ms + bwd_ms) / 1e3),
           "roofline": {"kernel": "k_smp_rows_a / k_smp_rows_b (entries grouped by block index)", "bound": "l2",
                        "hbm_bytes_per_fwd": hbm, "l2_row_bytes_per_fwd": l2,
                        "l2_gbs_fwd": l2 / (fwd_ms / 1e3) / 1e9, "l2_gbs_bwd": 2 * l2 / (bwd_ms / 1e3) / 1e9,
                        "hbm_frac_fwd": hbm / (fwd_ms / 1e3) / 1e9 / pk["hbm_gbs"]}}
    t.close()
    del x, idx
    torch.cuda.empty_cache()
    if budget:
        res["cpu_baseline"] = cpu_pair("sampled", "grad128", budget)
    return res


# ----------------------------------------------------------------------------- oracle
def oracle_sample(w, corr):
    """The CPU oracle's bounded sample: the sub-tensor i_4 < 10 of the workload."""
    from oracle import trd_oracle as O
    from paper_2305_09044_gb300 import synth
    dims = list(w.dims)
    sub = dims[:-1] + [ORACLE_SLICES]
    truth = synth.gaussian_cores(w.dims, w.ranks, w.data_seed)
    truth_sub = [Z if k < len(dims) - 1 else Z[:, :ORACLE_SLICES, :] for k, Z in enumerate(truth)]
    Xt = O.reconstruct_unfold(truth_sub)
    if corr is None:
        corr = synth.draw_corruption(w)
    sl = (slice(None),) * (len(dims) - 1) + (slice(0, ORACLE_SLICES),)
    c = synth.Corruption(corr.mask[sl], corr.outlier[sl], corr.outlier_u[sl],
                         None if corr.noise is None else corr.noise[sl])
    X = synth.assemble(Xt, c).astype(np.float32).astype(np.float64)
    P = c.mask.astype(np.float64)
    cores = O.init_cores(w.dims, w.ranks, seed=w.init_seed)
    cores = [Z if k < len(dims) - 1 else Z[:, :ORACLE_SLICES, :] for k, Z in enumerate(cores)]
    obs = P > 0
    sigma = O.adaptive_sigma((X - O.reconstruct_unfold(cores))[obs], float(np.sqrt(np.mean(X[obs] ** 2))))
    return X, P, cores, sigma, sub


def cpu_baseline(w, corr, budget_s=15.0):
    from oracle import trd_oracle as O
    X, P, cores, sigma, sub = oracle_sample(w, corr)
    slots = int(np.prod(sub))
    done, spent, k = 0, 0.0, 0
    while spent < budget_s or done == 0:
        t0 = time.perf_counter()
        cores = O.core_update(X, P, cores, k % len(sub), sigma).cores
        spent += time.perf_counter() - t0
        done += 1
        k += 1
        if done >= 8:
            break
    return {"value": done * slots / spent, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{done} FP64 oracle core updates on the {'x'.join(map(str, sub))} sub-tensor "
                      f"(i_4 < {ORACLE_SLICES}) of the workload, {slots} slots each; numpy BLAS "
                      f"threads for the products, element-wise steps single-threaded",
            "seconds": spent}


def run_reference(args, rank, world):
    if rank != 0:
        return
    from paper_2305_09044_gb300 import synth
    from oracle import trd_oracle as O
    w = synth.WORKLOADS[WORKLOAD]
    X, P, cores, sigma, sub = oracle_sample(w, None)
    slots = int(np.prod(sub))
    N = len(sub)
    for i in range(max(args.warmup, 3)):
        cores = O.core_update(X, P, cores, i % N, sigma).cores
    t0 = time.perf_counter()
    for i in range(args.steps):
        cores = O.core_update(X, P, cores, i % N, sigma).cores
    dt = time.perf_counter() - t0
    value = args.steps * slots / dt
    cfg = workload_config(w, "fp64 (CPU oracle)")
    cfg["sample"] = f"each step is one oracle core update on the {'x'.join(map(str, sub))} sub-tensor"
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": dt * 1e3 / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": cfg,
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                            "sample": cfg["sample"]},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ----------------------------------------------------------------------------- dist helpers
_pg = None


def replica_workload(w, rank, world):
    """N > 1 runs independent replicas (the path does not shard): rank r solves its own
    problem, drawn with data and initialisation seeds offset by 100 r."""
    if world <= 1:
        return w
    import dataclasses
    return dataclasses.replace(w, data_seed=w.data_seed + 100 * rank, init_seed=w.init_seed + 100 * rank)


def job_throughput(world, slots_per_step, steps, ms_max):
    """Whole-job sampled entries per second: every rank's slots over the slowest rank's time."""
    return world * slots_per_step * steps / (ms_max / 1e3)


def _init_dist(world):
    global _pg
    if world > 1 and _pg is None:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("gloo")
        _pg = dist


def _barrier(world):
    if world > 1:
        _pg.barrier()


def _max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64)
    _pg.all_reduce(t, op=_pg.ReduceOp.MAX)
    return float(t.item())


def main():
    args = parse()
    if args.oracle_probe:
        oracle_probe_main(args.oracle_probe, args.oracle_budget)
        return
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.configs_only:
        import torch
        import __graft_entry__
        __graft_entry__.build()
        torch.cuda.set_device(local)
        if rank == 0:
            measured = measure_peaks(torch)
            print(json.dumps({"peaks_measured_here": measured, "configs": other_configs(args, torch, measured)}),
                  flush=True)
        return
    if args.video_rank80:
        import torch
        import __graft_entry__
        __graft_entry__.build()
        torch.cuda.set_device(local)
        if rank == 0:
            print(json.dumps({"video_rank80": video_rank80(torch, args.precision or "bf16")}), flush=True)
        return
    if args.image_only:
        import torch
        import __graft_entry__
        __graft_entry__.build()
        torch.cuda.set_device(local)
        prec = args.precision or "bf16"
        if rank == 0:
            print(json.dumps({"image": [image_quality(n, prec, torch) for n in ("image", "imagec")]}),
                  flush=True)
        return
    _init_dist(world)
    run_ours(args, rank, world, local)
    if world > 1:
        _pg.destroy_process_group()


if __name__ == "__main__":
    main()
