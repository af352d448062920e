#!/usr/bin/env python3
"""Throughput of batched Kerr geodesic integration on one GB300 (per rank).

Workload (one "step"): every ray of a 1024 x 1024 image plane, spin a = 0.99,
inclination 17 deg, observer at r = 1000 M, image plane +-25 M, integrated
backward to capture (r < 1.01 r_h) or escape (beyond its start radius) with
the FP32+Kahan persistent kernel at tolerance 1e-6.  Inputs are synthetic
(the camera specification; initial states are built on the device).

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on the host cores on bounded samples of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("rays/s to termination at ≤1e-5 rel. err (FP32 vs FP64 path); "
          "% of FP32 pipe peak")
UNIT = "rays/s"
# Algorithmic FLOPs, counted by the FLOP-counting transcription of eqs.
# opt0/opti in oracle/flops.py (tests/test_flops.py pins both numbers):
FLOPS_PER_RHS = 160          # one right-hand side
FLOPS_PER_ATTEMPT = 366      # stage sums, error norm and update of one attempt
FP32_LANES_PER_SM = 128      # FP32 FMA lanes per SM (one FMA = 2 FLOPs)
FP64_NOMINAL_TFLOPS = 1.25   # GB300 FP64 (non-tensor) nominal rate
WORKLOAD = ("camera 1024x1024, a=0.99, i=17deg, r_obs=1000M, +-25M, tol 1e-6, "
            "FP32+Kahan persistent kernel")
# The autotuner's cache file (per machine; a fresh GPU machine starts empty).
TUNE_CACHE = os.path.join(os.environ.get("TMPDIR", "/tmp"), "kerr_tune_cache.txt")


# Sources of the integrator kernels (the surrogate's files are left out:
# they do not change these kernels).
TRACE_SOURCES = ("kerr_math.cuh", "kerr_df.cuh", "kerr_trace.cuh", "kerr_variants.h",
                 "kerr_trace_f32.cu", "kerr_trace_f32b.cu", "kerr_trace_zone.cu",
                 "kerr_trace_f64.cu")


def kernel_source_hash() -> str:
    """Hash of the integrator's CUDA sources: ncu counters are only valid for
    the kernels they were taken from."""
    import hashlib
    d = os.path.join(ROOT, "paper_1706_07062_gb300", "csrc")
    h = hashlib.sha256()
    for f in TRACE_SOURCES:
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def load_traffic() -> dict:
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum)
    from the committed ncu summary, if it was taken from the current kernels."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return {}
    with open(p) as fh:
        t = json.load(fh)
    if t.get("source_hash") != kernel_source_hash():
        return {}
    return t.get("bytes_per_launch", {})


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.rows = []
        self.proc = None
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "100"]
        if uuid:
            cmd += ["-i", uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except OSError:
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.th.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in self.rows for j in range(4)
                          if r[5 + j].lower().startswith("active")})
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": reasons, "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def reduce_step_time(ms: float, device=None) -> float:
    """The job's time per step: the maximum over ranks when a process group
    is up (one rank per GPU; replicas, so this is the only collective), else
    the local time.  `device`: where the reduction tensor lives (the rank's
    GPU for NCCL, the CPU for gloo)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def measure_alu_peaks(K, dev, stream, target_ms: float = 150.0) -> dict:
    """Measured FP32 and FP64 pipe rates of this GPU: the FMA-chain kernel
    (kerr_fma_chain) timed with CUDA events on `stream`, best of three
    launches of ~target_ms each, with the SM clock sampled meanwhile."""
    import torch
    props = torch.cuda.get_device_properties(dev)
    bps = 4
    sink = torch.empty(props.multi_processor_count * bps * 256, dtype=torch.float32, device=dev)
    uuid = None
    try:
        uuid = "GPU-" + str(props.uuid)
    except Exception:
        uuid = None
    out = {}
    for name, kind, guess in (("fp32", K.PEAK_FP32, 70.0), ("fp32x2", K.PEAK_FP32X2, 70.0),
                              ("fp64", K.PEAK_FP64, 1.2)):
        # size the launch from a nominal guess, then from a first measurement
        rounds = max(16, int(guess * 1e12 * target_ms * 1e-3
                             / (2 * props.multi_processor_count * bps * 256 * 128)))
        K.kerr_fma_chain(kind, 16, sink, bps, stream=stream)
        sampler = ClockSampler(uuid)
        best = None
        for _ in range(4):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fl = K.kerr_fma_chain(kind, rounds, sink, bps, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            tf = fl / (e0.elapsed_time(e1) * 1e-3) / 1e12
            best = tf if best is None else max(best, tf)
        clk = sampler.stop()
        out[name] = {"tflops": round(best, 3), "clocks": clk}
    return out


def job_throughput(units_per_rank: int, world: int, ms_per_step: float) -> float:
    """Whole-job units per second: every rank processes its own units
    (weak scaling) in at most ms_per_step."""
    return world * units_per_rank / (ms_per_step * 1e-3)


def run_ours(args, rank, world, local_rank):
    import torch

    from paper_1706_07062_gb300 import kerr as K
    from paper_1706_07062_gb300 import workloads as W

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    from paper_1706_07062_gb300 import shard

    spec = W.CAMERA_1024
    cam = K.camera(*spec.as_tuple())
    n_total = spec.n
    prec = K.FP64 if args.prec == "fp64" else K.FP32_KAHAN
    ctx = K.kerr_init(spec.a)
    opts = K.default_opts(prec=prec, tol=W.TOL_1024)
    if args.autotune:
        opts.variant = K.kerr_autotune(ctx, cam, opts, sample=1 << 16)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    # one image; with several ranks each traces its interleaved rows of it
    # (the outputs would be concatenated on the host; no exchange on the GPU)
    if world > 1:
        my_pix = torch.from_numpy(shard.row_partition(spec.nx, spec.ny, world, rank)).to(dev)
        n = int(my_pix.numel())
    else:
        my_pix, n = None, n_total
    out = K.alloc_out(n, dev)

    def step(o=None):
        o = o or out
        if my_pix is None:
            K.kerr_trace_camera(ctx, cam, opts, out=o, stream=stream)
        else:
            K.kerr_trace_camera_pixels(ctx, cam, my_pix, opts, out=o, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)

    # ---- timed region: K steps, L2 flushed between steps (outside the events)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    kern_ms, phase_ms, rhs32, rhs64, att, att64 = [], [], 0, 0, 0, 0
    rhs32z, att32z = 0, 0
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        uuid = None
    sampler = ClockSampler(uuid) if rank == 0 else None
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    t_wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
        s = K.kerr_get_stats(ctx)          # synchronises the library stream
        kern_ms.append(s.kernel_ms)
        phase_ms.append(list(s.phase_ms))
        rhs32 += s.rhs_fp32
        rhs64 += s.rhs_fp64
        att += s.attempts
        att64 += s.attempts_fp64
        rhs32z += s.rhs_fp32_zone_phase
        att32z += s.attempts_fp32_zone_phase
    torch.cuda.synchronize(dev)
    if dist is not None:
        dist.barrier()
    t_wall = time.perf_counter() - t_wall0
    clocks = sampler.stop() if sampler else None
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = reduce_step_time(sum(step_ms) / len(step_ms), dev if dist is not None else None)
    value = n_total / (ms * 1e-3)
    stats = K.kerr_get_stats(ctx)

    # ---- rooflines (algorithmic FLOPs from the counted right-hand sides),
    # each phase's FLOPs divided by that phase's own time
    att32 = att - att64
    fl32 = rhs32 * FLOPS_PER_RHS + att32 * FLOPS_PER_ATTEMPT
    fl32z = rhs32z * FLOPS_PER_RHS + att32z * FLOPS_PER_ATTEMPT   # FP32 steps of the zone phase
    fl32s = fl32 - fl32z                                          # FP32 stepping phase
    fl64 = rhs64 * FLOPS_PER_RHS + att64 * FLOPS_PER_ATTEMPT
    kms = sum(kern_ms) / len(kern_ms)
    ph = [sum(p[i] for p in phase_ms) / len(phase_ms) for i in range(4)]
    peaks, peak_src = load_peaks()
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    nominal32 = sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    alu = measure_alu_peaks(K, dev, stream) if rank == 0 and not args.skip_alu_peaks else None
    if alu:
        peak32 = max(alu["fp32"]["tflops"], alu["fp32x2"]["tflops"])
        peak64 = alu["fp64"]["tflops"]
        src32 = (f"measured: FMA-chain kernel (kerr_fma_chain) in this run, best of fma.f32 "
                 f"and fma.f32x2 (of measured; nominal {sms} SMs x {FP32_LANES_PER_SM} lanes "
                 f"x 2 x {sm_max:.0f} MHz = {nominal32:.1f})")
        src64 = "measured: FMA-chain kernel (kerr_fma_chain, fma.f64) in this run (of measured)"
    else:
        peak32, peak64 = nominal32, FP64_NOMINAL_TFLOPS
        src32 = f"nominal {sms} SMs x {FP32_LANES_PER_SM} lanes x 2 x {sm_max:.0f} MHz"
        src64 = "nominal GB300 FP64 rate"
    traffic = load_traffic()
    if prec == K.FP32_KAHAN:
        t32, t64 = ph[1], ph[2]
        ach32 = fl32s / args.steps / (t32 * 1e-3) / 1e12 if t32 > 0 else 0.0
        ach64 = fl64 / args.steps / (t64 * 1e-3) / 1e12 if t64 > 0 else 0.0
        fp32_roof = {"kernel": "trace_f32_kernel (FP32 stepping phase)", "bound": "alu",
                     "achieved": round(ach32, 3), "peak": round(peak32, 2), "unit": "TFLOP/s",
                     "frac": round(ach32 / peak32, 4), "kernel_ms": round(t32, 4),
                     "traffic": traffic.get("fp32_stepping"), "peak_source": src32,
                     "frac_of_nominal": round(ach32 / nominal32, 4)}
        zone_roof = {"kernel": "trace_f32_kernel (FP64 zone phase)", "bound": "alu",
                     "achieved": round(ach64, 4), "peak": round(peak64, 4), "unit": "TFLOP/s",
                     "frac": round(ach64 / peak64, 4), "kernel_ms": round(t64, 4),
                     "traffic": traffic.get("fp64_zone"), "peak_source": src64,
                     "frac_of_nominal": round(ach64 / FP64_NOMINAL_TFLOPS, 4),
                     "fp32_flops_of_zone_phase": fl32z // args.steps}
        dominant = zone_roof if t64 > t32 else fp32_roof
        roofline = dict(dominant)
        roofline["phase_ms"] = {"setup": round(ph[0], 4), "fp32_stepping": round(ph[1], 4),
                                "fp64_zone": round(ph[2], 4), "finish": round(ph[3], 4)}
        roofline["fp32_stepping"] = fp32_roof
        roofline["fp64_zone"] = zone_roof
    else:
        ach64 = fl64 / args.steps / (kms * 1e-3) / 1e12
        roofline = {"kernel": "trace_f64_kernel", "bound": "alu", "achieved": round(ach64, 4),
                    "peak": round(peak64, 4), "unit": "TFLOP/s", "frac": round(ach64 / peak64, 4),
                    "kernel_ms": round(kms, 4), "traffic": traffic.get("fp64_path"),
                    "peak_source": src64}
    roofline["attempts_per_ray"] = round(att / args.steps / n, 2)
    roofline["fp64_attempt_share"] = round(att64 / max(att, 1), 4)
    roofline["fp32_flops_per_step"] = fl32 // args.steps
    if alu:
        roofline["alu_peaks_measured"] = alu
    roofline["fp64_flops_per_step"] = fl64 // args.steps

    result = {"metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
              "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
              "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
              "dtype": "f32" if prec == K.FP32_KAHAN else "f64", "data": "synthetic",
              "config": {"workload": WORKLOAD if prec == K.FP32_KAHAN else
                         WORKLOAD.replace("FP32+Kahan", "FP64"),
                         "rays": n_total, "rays_per_gpu": n,
                         "parallelism": ("one image" if world == 1 else
                                         f"image rows interleaved over {world} processes"),
                         "l2": "flushed between steps (512 MiB write, outside the events)",
                         "variant": stats.variant},
              "gpu_launches": args.steps * (4 if prec == K.FP32_KAHAN else 1),
              "roofline": roofline, "clocks": clocks,
              "timed_wall_s": round(t_wall, 3)}

    # ---- end to end through the C ABI with host (pinned) buffers: every rank
    # its share, the job's time the slowest rank's
    if not args.skip_e2e:
        host = K.alloc_out(n, device="cpu", pinned=True)
        for _ in range(2):
            step(host)
        e2e_t = []
        for _ in range(max(3, min(args.steps, 10))):
            flush.zero_()
            torch.cuda.synchronize(dev)
            if dist is not None:
                dist.barrier()
            t0 = time.perf_counter()
            step(host)                     # returns once the host buffers hold the results
            e2e_t.append(time.perf_counter() - t0)
        e2e_ms = reduce_step_time(1e3 * sum(e2e_t) / len(e2e_t),
                                  dev if dist is not None else None)
        # inputs: the camera (56 bytes) and, split across ranks, the pixel list
        h2d = 56 + (8 * n if my_pix is not None else 0)
        result["e2e"] = {"value": round(n_total / (e2e_ms * 1e-3), 1), "unit": UNIT,
                         "h2d_bytes_per_step": h2d,
                         "d2h_bytes_per_step": n * (8 * 8 + 4 + 4 + 4 * 4)}

    # ---- FP32+Kahan without the FP64 zone (comparison leg)
    if rank == 0 and prec == K.FP32_KAHAN and not args.skip_fp64:
        onz = K.default_opts(prec=K.FP32_KAHAN, tol=W.TOL_1024, fp64_zone=0.0)
        outnz = K.alloc_out(n_total, dev)
        K.kerr_trace_camera(ctx, cam, onz, out=outnz, stream=stream)
        torch.cuda.synchronize(dev)
        tnz = []
        for _ in range(3):
            flush.zero_()
            a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a_.record(stream)
            K.kerr_trace_camera(ctx, cam, onz, out=outnz, stream=stream)
            b_.record(stream)
            torch.cuda.synchronize(dev)
            tnz.append(a_.elapsed_time(b_))
        result["fp32_no_zone"] = {"value": round(n_total / (min(tnz) * 1e-3), 1), "unit": UNIT,
                                  "ms_per_step": round(min(tnz), 3),
                                  "note": "same path with fp64_zone = 0 (every step FP32+Kahan)"}
        result["_nz_out"] = outnz

    # ---- FP32+Kahan with float-float zone steps (comparison leg): the zone's
    # steps in ~48-bit float-float arithmetic on the FP32 pipe instead of FP64
    if rank == 0 and prec == K.FP32_KAHAN and not args.skip_fp64:
        odf = K.default_opts(prec=K.FP32_KAHAN, tol=W.TOL_1024, zone_prec=K.ZONE_F32X2)
        outdf = K.alloc_out(n_total, dev)
        K.kerr_trace_camera(ctx, cam, odf, out=outdf, stream=stream)
        torch.cuda.synchronize(dev)
        tdf, zdf = [], []
        for _ in range(3):
            flush.zero_()
            a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a_.record(stream)
            K.kerr_trace_camera(ctx, cam, odf, out=outdf, stream=stream)
            b_.record(stream)
            torch.cuda.synchronize(dev)
            tdf.append(a_.elapsed_time(b_))
            zdf.append(K.kerr_get_stats(ctx).phase_ms[2])
        result["fp32_zone_float_float"] = {
            "value": round(n_total / (min(tdf) * 1e-3), 1), "unit": UNIT,
            "ms_per_step": round(min(tdf), 3), "zone_phase_ms": round(min(zdf), 3),
            "note": "same path with zone_prec = KERR_ZONE_F32X2: steps inside 1.5 r_h in "
                    "float-float (~48-bit) arithmetic on the FP32 pipe instead of FP64"}
        result["_df_out"] = outdf

    # ---- plain FP64 GPU path on the same workload (comparison leg)
    if rank == 0 and prec == K.FP32_KAHAN and not args.skip_fp64:
        o64 = K.default_opts(prec=K.FP64, tol=W.TOL_1024)
        out64 = K.alloc_out(n_total, dev)
        K.kerr_trace_camera(ctx, cam, o64, out=out64, stream=stream)
        torch.cuda.synchronize(dev)
        t64 = []
        for _ in range(2):
            flush.zero_()
            a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a_.record(stream)
            K.kerr_trace_camera(ctx, cam, o64, out=out64, stream=stream)
            b_.record(stream)
            torch.cuda.synchronize(dev)
            t64.append(a_.elapsed_time(b_))
        result["fp64_path"] = {"value": round(n_total / (min(t64) * 1e-3), 1), "unit": UNIT,
                               "ms_per_step": round(min(t64), 3)}
        result["_fp64_out"] = out64

    # ---- learned surrogate: train on integrator rays, render with fallback
    if rank == 0 and not args.skip_surrogate:
        result["surrogate"] = run_surrogate(args, K, W, dev, stream)
        result["_surr_img"] = result["surrogate"].pop("_img0")

    # ---- the other workloads: 64 uneven images in one launch, 2^20 particles
    if rank == 0 and not args.skip_batch:
        result["batch64"] = run_batch64(K, W, dev, stream)
    if rank == 0 and not args.skip_particles:
        result["particles"] = run_particles(K, W, dev, stream)

    # ---- paper-mode fixed-step benchmark (the paper's own timing setting)
    if rank == 0 and not args.skip_paper_mode:
        result["paper_mode"] = run_paper_mode(K, dev, stream)

    # ---- CPU baseline: the oracle on the host cores (rank 0, N = 1 only)
    if rank == 0 and world == 1 and not args.skip_cpu:
        result["cpu_baseline"], acc = cpu_baseline(spec, W, out, result.get("_fp64_out"),
                                                   result.get("_nz_out"),
                                                   result.get("_surr_img"),
                                                   result.get("_df_out"))
        if acc:
            result["accuracy"] = acc
    result.pop("_fp64_out", None)
    result.pop("_nz_out", None)
    result.pop("_df_out", None)
    result.pop("_surr_img", None)
    if rank == 0:
        print(json.dumps(result), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    ctx.close()


# Algorithmic FLOPs of one surrogate forward pass (unpadded widths
# 4 -> 256 -> 256 -> 256 -> 256 -> 8, one multiply-add = 2 FLOPs); a training
# sample costs three times that (forward, input gradients, weight gradients).
SURR_FWD_FLOPS = 2 * (4 * 256 + 3 * 256 * 256 + 256 * 8)


def run_surrogate(args, K, W, dev, stream):
    """Config: surrogate trained on integrator-generated rays (alpha, beta ~
    U[-25, 25], a ~ U[0, 0.998], i ~ U[5, 85] deg), evaluated on 2048 x 2048
    images with integrator fallback (capture probability in [0.05, 0.95] or
    within 0.5 M of the critical curve).  Reports rays/s of surrogate plus
    fallback, the integrator alone on the same images, and the disagreement
    and label errors against the FP64 integrator (itself pinned to the
    oracle at 1e-9)."""
    import torch

    ctx = K.kerr_init(0.5)
    opts = K.default_opts()                       # FP32+Kahan, tol 1e-6
    pts = torch.from_numpy(W.surrogate_points(args.surrogate_rays)).to(dev)
    torch.cuda.synchronize(dev)

    def timed(fn):
        a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a_.record(stream)
        r = fn()
        b_.record(stream)
        torch.cuda.synchronize(dev)
        return r, a_.elapsed_time(b_) * 1e-3

    (inp, tgt, msk), t_lab = timed(lambda: K.kerr_surrogate_targets(
        ctx, pts, 1000.0, opts, stream=stream))
    del pts
    net = K.Surrogate(W.surrogate_init())
    losses, t_tr = timed(lambda: K.kerr_surrogate_train(
        net, inp, tgt, msk, epochs=args.surrogate_epochs, batch=8192, lr=2e-3, stream=stream))
    n_train = int(inp.shape[0])
    del inp, tgt, msk

    # the fused forward alone on one 2048 x 2048 image's rows (seeded inputs
    # in the network's input ranges, resident in HBM; best of 5 calls)
    n_fwd = 2048 * 2048
    gen = torch.Generator(device=dev).manual_seed(2048)
    lo = torch.tensor([-1.0, -1.0, 0.0, 0.1], device=dev)
    hi = torch.tensor([1.0, 1.0, 0.998, 1.0], device=dev)
    x_fwd = lo + (hi - lo) * torch.rand((n_fwd, 4), device=dev, generator=gen)
    o_fwd = torch.empty((n_fwd, 8), device=dev)
    K.kerr_surrogate_forward(net, x_fwd, out=o_fwd, stream=stream)
    t_fwd = min(timed(lambda: K.kerr_surrogate_forward(net, x_fwd, out=o_fwd, stream=stream))[1]
                for _ in range(5))
    del x_fwd, o_fwd
    peaks, peaks_src = load_peaks()

    o64 = K.default_opts(prec=K.FP64)
    t_sur = t_int = 0.0
    n_tot = n_fb = 0
    dis = dis_n = 0
    # the same renders with the fallback rays' zone steps in float-float
    opts_df = K.default_opts(zone_prec=K.ZONE_F32X2)
    t_sur_df = 0.0
    errs = {k: [] for k in ("r1", "phi1", "r2", "phi2", "g1")}
    img0 = None
    for cs in W.surrogate_eval_cameras():
        cam = K.camera(*cs.as_tuple())
        n = cs.n
        K.kerr_surrogate_render(ctx, net, cam, opts, stream=stream)      # warm (graphs)
        ref32 = K.alloc_out(n, dev, diag=False, cross=True)
        K.kerr_trace_camera(ctx, cam, opts, out=ref32, stream=stream)
        torch.cuda.nvtx.range_push("surrogate_render")      # for profiler filters
        (out, fb, nfb), dt = timed(lambda: K.kerr_surrogate_render(ctx, net, cam, opts,
                                                                   stream=stream))
        torch.cuda.nvtx.range_pop()
        K.kerr_surrogate_render(ctx, net, cam, opts_df, stream=stream)   # warm
        _, dtd = timed(lambda: K.kerr_surrogate_render(ctx, net, cam, opts_df, stream=stream))
        t_sur_df += dtd
        _, dti = timed(lambda: K.kerr_trace_camera(ctx, cam, opts, out=ref32, stream=stream))
        ref = K.alloc_out(n, dev, diag=False, cross=True)
        K.kerr_trace_camera(ctx, cam, o64, out=ref, stream=stream)
        torch.cuda.synchronize(dev)
        t_sur += dt
        t_int += dti
        n_tot += n
        n_fb += nfb
        net_px = fb == 0
        cap_net = out[0] >= 0.5
        cap_ref = ref.status == 2
        dis += int((cap_net[net_px] != cap_ref[net_px]).sum())
        dis_n += int(net_px.sum())
        for j, key in enumerate(("r1", "phi1", "r2", "phi2", "g1")):
            a_, b_ = out[1 + j], ref.cross[j]
            ok = net_px & ~torch.isnan(a_) & ~torch.isnan(b_)
            if key.startswith("phi"):
                e = torch.remainder(a_[ok] - b_[ok] + math.pi, 2 * math.pi) - math.pi
                e = e.abs()
            elif key.startswith("r"):
                e = ((a_[ok] - b_[ok]) / b_[ok]).abs()
            else:
                e = (a_[ok] - b_[ok]).abs()
            errs[key].append(e.double().cpu().numpy())
        if img0 is None:      # kept for the CPU leg's comparison with the oracle
            img0 = {"spec": cs, "out": out.cpu().numpy(), "fallback": fb.cpu().numpy()}
        del out, fb, ref, ref32
    err = {}
    for key, v in errs.items():
        v = np.concatenate(v) if v else np.zeros(0)
        kind = "rel" if key.startswith("r") else "abs"
        err[key] = {"kind": kind, "n": int(v.size),
                    "median": float(np.median(v)) if v.size else None,
                    "p90": float(np.percentile(v, 90)) if v.size else None,
                    "p99": float(np.percentile(v, 99)) if v.size else None}
    ctx.close()
    v_sur = n_tot / t_sur
    v_int = n_tot / t_int
    ep = args.surrogate_epochs
    return {"_img0": img0, "value": round(v_sur, 1), "unit": UNIT,
            "workload": "8 images 2048x2048 (seeded a ~ U[0,0.998], i ~ U[5,85] deg), "
                        "r_obs 1000M, +-25M; fallback: p in [0.05,0.95] or within 0.5M of "
                        "the critical curve; integrator FP32+Kahan tol 1e-6",
            "integrator_only": round(v_int, 1), "gain": round(v_sur / v_int, 3),
            "value_fallback_float_float_zone": round(n_tot / t_sur_df, 1),
            "fallback_frac": round(n_fb / n_tot, 5),
            "capture_disagreement": dis / max(dis_n, 1),
            "reference": "GPU FP64 integrator, tol 1e-6, same images",
            "errors_on_network_pixels": err,
            "forward": {"rows": n_fwd, "ms": round(t_fwd * 1e3, 3),
                        "tflops": round(SURR_FWD_FLOPS * n_fwd / t_fwd / 1e12, 1),
                        "frac_bf16_burst": round(SURR_FWD_FLOPS * n_fwd / t_fwd / 1e12
                                                 / peaks["bf16_tflops"], 4),
                        "peak": peaks_src,
                        "kernel": "mlp_forward_tc_kernel (all five layers, two 128-row "
                                  "tiles in flight per CTA)"},
            "train": {"rays": n_train, "epochs": ep, "batch": 8192,
                      "label_s": round(t_lab, 3), "train_s": round(t_tr, 3),
                      "samples_per_s": round(n_train * ep / t_tr, 1),
                      "achieved_tflops": round(3 * SURR_FWD_FLOPS * n_train * ep / t_tr / 1e12,
                                               2),
                      "frac_bf16_sustained": round(
                          3 * SURR_FWD_FLOPS * n_train * ep / t_tr / 1e12
                          / peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"]), 4),
                      "kernels": "fused: chain (forward, loss, backward data per 128-row "
                                 "tile), batch-contracted weight gradients, Adam",
                      "loss_first_last": [float(losses[0]), float(losses[-1])]}}


def run_batch64(K, W, dev, stream):
    """64 images with sides drawn from {128, ..., 2048}, spins U[0, 0.998],
    inclinations U[5, 85] deg (seed 1708; 34.9 M rays) traced in one captured
    launch, FP32+Kahan, tol 1e-6: latency of the launch and rays/s."""
    import torch

    specs = W.camera_batch()
    cams = [K.camera(*c.as_tuple()) for c in specs]
    n = sum(c.n for c in specs)
    ctx = K.kerr_init(0.0)
    opts = K.default_opts(tol=1e-6)
    # the autotuner picks the launch configuration on a 2^18-ray sample of the
    # batch (kept for the context's later calls; cached per GPU and workload)
    t0 = time.perf_counter()
    tuning = K.kerr_autotune_cameras(ctx, cams, opts, sample=1 << 18, cache_path=TUNE_CACHE,
                                     stream=stream)
    tune_s = time.perf_counter() - t0
    out = K.alloc_out(n, dev, diag=False)
    K.kerr_trace_camera(ctx, cams, opts, out=out, stream=stream)      # warm (graph, buffers)
    torch.cuda.synchronize(dev)
    times = []
    for _ in range(2):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        K.kerr_trace_camera(ctx, cams, opts, out=out, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        times.append(e0.elapsed_time(e1))
    s = K.kerr_get_stats(ctx)
    st = torch.bincount(out.status.long(), minlength=8).tolist()
    ctx.close()
    ms = min(times)
    return {"workload": "64 images, sides U{128..2048}, a ~ U[0,0.998], i ~ U[5,85] deg, "
                        "r_obs 1000M, +-25M, seed 1708, one launch, FP32+Kahan tol 1e-6",
            "rays": n, "latency_ms": round(ms, 2), "value": round(n / (ms * 1e-3), 1),
            "unit": UNIT, "phase_ms": [round(x, 2) for x in s.phase_ms],
            "attempts_per_ray": round(s.attempts / n, 2), "status_count": st,
            "autotune": dict(tuning.as_dict(), seconds=round(tune_s, 2), used=s.variant)}


def run_particles(K, W, dev, stream):
    """2^20 bound particles, a = 0.7 (seed 1707): semi-major axes log-uniform
    in [10, 1000] M, e ~ U[0, 0.9], isotropic planes, 100 Newtonian radial
    periods each (or capture); FP32+Kahan and the FP64 path on all of them,
    tol 1e-6, with the launch configuration picked by the autotuner (on a
    sample run for a tenth of the time: 2^18 particles in FP32, 2^16 in FP64,
    many more than the GPU has lanes, as in the full run).  Particles/s,
    attempted steps/s, and the drift of the constants of motion E, L_z and
    Carter's Q between start and end (end points after 100 periods are not
    determined to 1e-5 by the method: orbital phase error grows with every
    period, so the constants are the accuracy measure here)."""
    import torch

    ps = W.particles()
    m = ps.x0.shape[1]
    ctx = K.kerr_init(ps.a)
    x0 = torch.tensor(ps.x0, device=dev).contiguous()
    v0 = torch.tensor(ps.v0, device=dev).contiguous()
    te = torch.tensor(ps.t_end, device=dev).contiguous()
    # constants of motion at the start (zero-step trace)
    start = K.alloc_out(m, dev)
    K.kerr_trace_particles(ctx, x0, v0, te, K.default_opts(prec=K.FP64, max_steps=0,
                                                           r_escape=-1.0),
                           out=start, stream=stream)
    torch.cuda.synchronize(dev)
    c0 = start.diag.double()
    scale = torch.stack([c0[0].abs(), c0[1].abs() + 1e-3,
                         c0[2] + (c0[1] - ps.a * c0[0]) ** 2])      # E, L_z, Carter's K
    res = {}
    for name, prec in (("fp32_kahan", K.FP32_KAHAN), ("fp64", K.FP64)):
        opts = K.default_opts(prec=prec, tol=1e-6, r_escape=-1.0)
        t0 = time.perf_counter()
        tuning = K.kerr_autotune_particles(ctx, x0, v0, te * 0.1, opts,
                                           sample=1 << (18 if prec == K.FP32_KAHAN else 16),
                                           cache_path=TUNE_CACHE, stream=stream)
        tune_s = time.perf_counter() - t0
        out = K.alloc_out(m, dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        K.kerr_trace_particles(ctx, x0, v0, te, opts, out=out, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        s = K.kerr_get_stats(ctx)
        steps = out.steps.double()
        ended = out.status == K.ENDTIME
        drift = {}
        for j, key in enumerate(("E", "Lz", "Q")):
            d = ((out.diag[j].double() - c0[j]).abs() / scale[j])[ended]
            q = torch.quantile(d, torch.tensor([0.5, 0.9, 0.99], dtype=torch.float64, device=dev))
            drift[key] = {"median": float(q[0]), "p90": float(q[1]), "p99": float(q[2])}
        res[name] = {"particles": m, "ms": round(ms, 2),
                     "value": round(m / (ms * 1e-3), 1), "unit": "particles/s",
                     "attempts_per_s": round(s.attempts / (ms * 1e-3), 1),
                     "steps_min_median_max": [int(steps.min()), float(steps.median()),
                                              int(steps.max())],
                     "status_count": list(s.status_count),
                     "drift_of_constants": drift,
                     "autotune": dict(tuning.as_dict(), seconds=round(tune_s, 2),
                                      used=s.variant)}
    ctx.close()
    res["workload"] = ("2^20 particles, a=0.7, A log-uniform [10,1000]M, e ~ U[0,0.9], isotropic, "
                       "100 radial periods, tol 1e-6, seed 1707")
    res["drift_note"] = ("|constant(end) - constant(start)| / scale over particles that reach "
                         "their end time; scale |E|, |L_z| + 1e-3, and Carter's K = Q + "
                         "(L_z - a E)^2 for Q")
    return res


# The paper's Titan Black entries of its Table 2 (ns per RK4 step per ray,
# OpenCL; other hardware: context, not a target).
PAPER_NS_PER_STEP = {("KS", "f32", "soa"): 0.309, ("KS", "f32", "aos"): 0.297,
                     ("KS", "f64", "soa"): 1.15, ("KS", "f64", "aos"): 1.15,
                     ("BL", "f32", "soa"): 0.175, ("BL", "f32", "aos"): 0.167,
                     ("BL", "f64", "soa"): 1.66, ("BL", "f64", "aos"): 1.65}


def run_paper_mode(K, dev, stream):
    """Sec. 4.2 setting: images of 64^2 .. 1024^2 rays from r = 1024 M toward
    a = 0.999 (inclination 60 deg and image plane +-20 M: this reading), each
    ray 1024 fixed RK4 steps of h = 1 in one launch, no termination; ns per
    RK4 step per ray = launch time / (1024 N), best over the image sizes, for
    KS / BL coordinates, FP32 / FP64 and SoA / AoS state layouts.  Initial states are built on the
    device (a zero-step camera trace); each timed launch starts from them
    (restored outside the events)."""
    import torch

    a, nsteps, h = 0.999, 1024, 1.0
    ctx = K.kerr_init(a)
    coords_rows = (("ks", "KS"), ("bl", "BL"))
    o0 = K.default_opts(prec=K.FP64, max_steps=0)
    rows = []
    best = {}
    for side in (64, 128, 256, 512, 1024):
        n = side * side
        cam = K.camera(a, math.radians(60.0), 1024.0, 20.0, side, side)
        out = K.alloc_out(n, dev, diag=False)
        K.kerr_trace_camera(ctx, cam, o0, out=out, stream=stream)
        torch.cuda.synchronize(dev)
        y_ks = torch.cat([out.x, out.k], 0).contiguous()        # (8, n) float64
        y_bl = K.kerr_bl_camera_states(cam, device=dev, stream=stream)
        torch.cuda.synchronize(dev)
        for coords, cname in coords_rows:
            y0 = y_ks if coords == "ks" else y_bl
            precs = [("f32", torch.float32, False), ("f64", torch.float64, False)]
            if coords == "ks":
                precs.append(("f32x2", torch.float32, True))   # two geodesics per thread
            for prec, dt, paired in precs:
                for lay, lid in (("soa", K.LAYOUT_SOA), ("aos", K.LAYOUT_AOS)):
                    init = y0.to(dt) if lid == K.LAYOUT_SOA else y0.T.contiguous().to(dt)
                    work = init.clone()
                    K.kerr_rk4_fixed(a, work, nsteps, h, layout=lid, stream=stream,
                                     coords=coords, paired=paired)               # warm-up
                    times = []
                    for _ in range(2):
                        work.copy_(init)
                        e0 = torch.cuda.Event(enable_timing=True)
                        e1 = torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        K.kerr_rk4_fixed(a, work, nsteps, h, layout=lid, stream=stream,
                                         coords=coords, paired=paired)
                        e1.record(stream)
                        torch.cuda.synchronize(dev)
                        times.append(e0.elapsed_time(e1))
                    ns = min(times) * 1e6 / (nsteps * n)
                    rows.append({"side": side, "coords": cname, "prec": prec, "layout": lay,
                                 "ns_per_step": round(ns, 5)})
                    key = (cname, prec, lay)
                    if key not in best or ns < best[key]["ns_per_step"]:
                        best[key] = {"ns_per_step": round(ns, 5), "side": side}
        del out, y_ks, y_bl
    ctx.close()
    summary = {}
    for (cname, prec, lay), b in sorted(best.items()):
        paper = PAPER_NS_PER_STEP[(cname, prec.replace("x2", ""), lay)]
        summary[f"{cname}_{prec}_{lay}"] = {
            "ns_per_step": b["ns_per_step"], "best_side": b["side"],
            "ray_steps_per_s": round(1e9 / b["ns_per_step"], 1),
            "paper_titan_black_ns": paper, "ratio_vs_paper": round(paper / b["ns_per_step"], 2)}
    return {"workload": "a=0.999, r_obs=1024M, i=60deg, +-20M, images 64^2..1024^2, "
                        "1024 fixed RK4 steps of h=1 per launch, no termination",
            "unit": "ns per RK4 step per ray (best over image sizes)",
            "best": summary, "all": rows}


def cpu_baseline(spec, W, out_gpu, out64, out_nz=None, surr_img=None, out_df=None):
    """Time the FP64 CPU oracle on a bounded seeded sample of the same image
    (all host cores), and use that same sample to state the GPU path's
    end-point error against it."""
    from oracle import oracle as O

    nthreads = os.cpu_count() or 1
    idx = W.camera_subset(spec)                       # seeded 4096-ray subset
    y0 = O.camera_ic(spec.a, spec.incl, spec.r_obs, spec.half_width, spec.nx, spec.ny, idx)
    oo = O.Opts(tol=W.TOL_1024)
    t0 = time.perf_counter()
    ref = O.trace(spec.a, y0, oo, nthreads=nthreads)
    dt = time.perf_counter() - t0
    n_done = len(idx)
    # extend the sample with more seeded rays to about 10 s of CPU work
    extra = int(min(200_000, max(0, (10.0 - dt) * n_done / dt)))
    if extra > 0:
        rng = np.random.default_rng(1706 + 1)
        idx2 = np.sort(rng.choice(spec.n, size=extra, replace=False))
        y2 = O.camera_ic(spec.a, spec.incl, spec.r_obs, spec.half_width, spec.nx, spec.ny, idx2)
        t1 = time.perf_counter()
        O.trace(spec.a, y2, oo, nthreads=nthreads)
        dt += time.perf_counter() - t1
        n_done += extra
    base = {"value": round(n_done / dt, 1), "unit": UNIT, "cores": nthreads, "kind": "oracle",
            "sample": f"{n_done} rays of the 1024x1024 image (seeded 4096-ray subset plus "
                      f"{extra} seeded random rays), FP64 oracle, tol 1e-6, {dt:.1f} s"}
    # one core, on the first 512 rays of the seeded subset
    t1 = time.perf_counter()
    O.trace(spec.a, y0[:512], oo, nthreads=1)
    base["single_core"] = {"value": round(512 / (time.perf_counter() - t1), 1), "unit": UNIT,
                           "sample": "first 512 rays of the seeded 4096-ray subset"}
    # accuracy of the GPU paths on the seeded subset
    acc = None
    try:
        flags = O.ill_conditioned(spec.a, y0, oo, ref=ref, rel=1e-5, nthreads=nthreads)

        def errs(o):
            x = o.x.cpu().numpy()[:, idx].T
            k = o.k.cpu().numpy()[:, idx].T
            st = o.status.cpu().numpy()[idx]
            ex = (np.linalg.norm(x[:, 1:4] - ref.y[:, 1:4], axis=1)
                  / np.linalg.norm(ref.y[:, 1:4], axis=1))
            ek = np.linalg.norm(k - ref.y[:, 4:8], axis=1) / np.linalg.norm(ref.y[:, 4:8], axis=1)
            e = np.maximum(ex, ek)
            g = ~flags
            return {"max_rel_err_well_conditioned": float(e[g].max()),
                    "median_rel_err": float(np.median(e)),
                    "p99_rel_err": float(np.quantile(e, 0.99)),
                    "frac_le_1e-5_all": float(np.mean(e <= 1e-5)),
                    "frac_le_1e-5_well_conditioned": float(np.mean(e[g] <= 1e-5)),
                    "status_mismatch_well_conditioned": int(np.sum((st != ref.status) & g))}
        acc = {"sample": len(idx), "reference": "FP64 CPU oracle, tol 1e-6",
               "ill_conditioned": int(flags.sum()), "fp32_kahan": errs(out_gpu)}
        if out64 is not None:
            acc["fp64"] = errs(out64)
        if out_nz is not None:
            # without the FP64 zone every step is an FP32 step: FP32 rounding
            # is modelled on the whole path when deciding what is determined
            flags = O.ill_conditioned(spec.a, y0, oo, ref=ref, rel=1e-5, nthreads=nthreads,
                                      noise_zone=0.0)
            acc["fp32_no_zone"] = dict(errs(out_nz), ill_conditioned=int(flags.sum()))
        if out_df is not None:
            acc["fp32_zone_float_float"] = errs(out_df)
    except Exception as exc:  # accuracy is a report, not the measurement
        acc = {"error": repr(exc)}
    if surr_img is not None:
        try:
            acc = acc or {}
            acc["surrogate"] = surrogate_vs_oracle(O, W, surr_img, nthreads)
        except Exception as exc:
            acc["surrogate"] = {"error": repr(exc)}
    return base, acc


def surrogate_vs_oracle(O, W, img, nthreads):
    """The surrogate's answers on a seeded 4096-pixel subset of the first
    evaluation image against the FP64 oracle (tol 1e-6, crossings on): capture
    disagreement and label errors on the pixels the network answered."""
    cs, out, fb = img["spec"], img["out"], img["fallback"]
    idx = W.camera_subset(cs, 4096, seed=1709)
    y0 = O.camera_ic(cs.a, cs.incl, cs.r_obs, cs.half_width, cs.nx, cs.ny, idx)
    ref = O.trace(cs.a, y0, O.Opts(tol=1e-6), nthreads=nthreads, crossings=True)
    net = fb[idx] == 0
    o = out[:, idx]
    res = {"sample": int(len(idx)), "network_pixels": int(net.sum()),
           "capture_disagreement": float(np.mean((o[0][net] >= 0.5) != (ref.status[net] == 2)))}
    for j, key in enumerate(("r1", "phi1", "r2", "phi2", "g1")):
        a_, b_ = o[1 + j], ref.cross[:, j]
        ok = net & ~np.isnan(a_) & ~np.isnan(b_)
        if key.startswith("phi"):
            e = np.abs(np.remainder(a_[ok] - b_[ok] + np.pi, 2 * np.pi) - np.pi)
        elif key.startswith("r"):
            e = np.abs(a_[ok] - b_[ok]) / b_[ok]
        else:
            e = np.abs(a_[ok] - b_[ok])
        res[key] = {"n": int(ok.sum()), "median": float(np.median(e)) if e.size else None,
                    "p99": float(np.percentile(e, 99)) if e.size else None}
    return res


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle as it stands, on host cores
# ---------------------------------------------------------------------------
def run_reference(args, rank, world):
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_1706_07062_gb300 import workloads as W

    spec = W.CAMERA_1024
    nthreads = os.cpu_count() or 1
    oo = O.Opts(tol=W.TOL_1024)
    rng = np.random.default_rng(4242)
    per_step = 2048

    def step():
        idx = np.sort(rng.choice(spec.n, size=per_step, replace=False))
        y0 = O.camera_ic(spec.a, spec.incl, spec.r_obs, spec.half_width, spec.nx, spec.ny, idx)
        t0 = time.perf_counter()
        O.trace(spec.a, y0, oo, nthreads=nthreads)
        return time.perf_counter() - t0

    for _ in range(args.warmup):
        step()
    ts = [step() for _ in range(args.steps)]
    ms = 1e3 * sum(ts) / len(ts)
    value = per_step / (ms * 1e-3)
    res = {"impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": UNIT,
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD.replace("FP32+Kahan persistent kernel",
                                                   "FP64 CPU oracle"),
                      "rays_per_step": per_step},
           "cpu_baseline": {"value": round(value, 1), "unit": UNIT, "cores": nthreads,
                            "kind": "oracle",
                            "sample": f"{per_step} seeded random rays of the 1024x1024 image "
                                      f"per step"},
           "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(res), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--prec", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--autotune", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-surrogate", action="store_true")
    ap.add_argument("--skip-paper-mode", action="store_true")
    ap.add_argument("--skip-batch", action="store_true")
    ap.add_argument("--skip-particles", action="store_true")
    ap.add_argument("--skip-alu-peaks", action="store_true",
                    help="rate the rooflines against nominal FP32/FP64 peaks instead of "
                         "measuring them with the FMA-chain kernel")
    ap.add_argument("--surrogate-rays", type=int, default=10_000_000)
    ap.add_argument("--surrogate-epochs", type=int, default=16)
    args = ap.parse_args()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        # one process per GPU: start them under torch.distributed.run
        launch = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
                  f"--nproc-per-node={args.gpus}", "--master-addr=127.0.0.1",
                  f"--master-port={29500 + os.getpid() % 1000}", os.path.abspath(__file__),
                  *sys.argv[1:]]
        os.execv(sys.executable, launch)
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        import __graft_entry__
        __graft_entry__.build()
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
