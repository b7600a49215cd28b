#!/usr/bin/env python
"""Benchmark: smoothed time-steps per second of the parallel MAP smoother.

Workload (one "step" = one complete MAP solve, elements -> filter scan -> RTS
pass -> x* written): the 2-D Wiener-velocity model (nx = 4, ny = 2, q = 1,
r = 0.1), dt = 1e-3, T = 2^20 intervals, FP32, seeded synthetic observations
resident in HBM.  The L2 cache (129 MB) is flushed by writing a 256 MiB buffer
before every timed step; each step is timed with CUDA events on the solve's
stream.  With --gpus N > 1 (torchrun) every rank solves its own independent
problem (replicas; the path has no cross-GPU exchange) and the value is the
total over ranks divided by the slowest rank's time.

--impl reference times the FP64 CPU oracle (sequential Kalman filter + RTS
smoother in plain C, one core) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("smoothed time-steps/sec at nx=4,T=2^20 (parallel vs sequential, same GB300) "
          "and % HBM roofline")
UNIT = "time-steps/s"
T_FULL = 2 ** 20
DT = 1e-3
WORKLOAD = "wiener-velocity 2-D (nx=4, ny=2, q=1, r=0.1), dt=1e-3, T=2^20, RTS smoother"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FP32_LANES_PER_SM, SMS, MAX_SM_MHZ = 128, 152, 2070.0


def model_and_data(seed, T=T_FULL):
    from paper_2512_13319_gb300 import synth
    model = synth.wiener_velocity(2, q=1.0, r=0.1)
    _, y = synth.simulate(model, T, DT, seed=seed, substeps=1)
    return model, y


# ----------------------------------------------------------------------------
# algorithmic work per step (multiply-adds; FLOP = 2 MAC) of each kernel of
# one solve, for state dimension n, measurement dimension m, K steps per
# thread, B threads per tile, nt tiles and process-noise rank r (r < n: the
# per-step update goes through the matrix inversion lemma)
# ----------------------------------------------------------------------------
def work_model(n, m, K, B, nt, wbytes, r=None):
    """Multiply-adds (returned as FLOP = 2 MAC) and minimal DRAM bytes per time
    step of each kernel of the linear-fold (LTI) solve, counted from the kernels:
    per-step work, plus the per-tile work (tile prefix, thread-prefix trees,
    tile map) spread over the B*K steps of a tile.  Redundant work of the
    shuffle reductions is not counted."""
    compose = n ** 3 + n ** 2                   # affine map composition
    apply_plain = 4.5 * n ** 3 + 2.5 * n ** 2   # one-variable combine (value function update)
    apply_alpha = 4.5 * n ** 3 + 4.5 * n ** 2   # ... plus the closed-loop map
    if r is not None and r < n:                 # matrix-inversion-lemma update of rank r
        apply_alpha = (n * n * r + n * r * (r + 1) / 2 + r ** 3 + r * n * n + r * r * n + n * n * r
                       + (2 * n * r + r * r + n * r + n * r)   # closed-loop offset g
                       + n ** 3 + n * n + n * n * (n + 1) / 2 + n * n)
    lin_node = 4 * n * n                        # (b, eta) tree node
    L = B * K
    mean_prefix_maps = (nt - 1) / 2.0           # tile maps a CTA folds, on average
    per_tile_down = (mean_prefix_maps * compose + n * n          # tile prefix
                     + 2 * (B - 1) * lin_node + B * apply_plain   # thread-prefix up/down sweeps, one combine each
                     + (B - 1) * compose)                         # tile map
    per_tile_rts = mean_prefix_maps * compose + (B - 1) * compose + B * n * n
    na = (r * n + n) if (r is not None and r < n) else (n * n + n)   # stored closed-loop map
    per_step_rts = (r * n + n * n + n * r) if (r is not None and r < n) else n * n
    mac = {
        "filter_reduce": 2 * n * m + ((B - 1) * lin_node + 2 * n * n) / L,
        "filter_down": n * m + apply_alpha + compose + per_tile_down / L,
        "rts_down": per_step_rts + per_tile_rts / L,
    }
    byt = {   # minimal DRAM bytes per step of each kernel
        "filter_reduce": wbytes * (m + 2 * n / K),
        "filter_down": wbytes * (m + 2 * n / K + na + (n * n + n) / K),
        "rts_down": wbytes * (na + (n * n + n) / K + n),
    }
    return {k: 2 * v for k, v in mac.items()}, byt


# DRAM bytes (read + write) of one k_filter_down launch on the nx=4, T=2^20 FP32
# workload, from one ncu capture of this kernel version (cold cache); None
# until the current version has been captured
K_FILTER_DOWN_DRAM_BYTES = 10482944 + 3812864
# the same for the single cooperative launch (k_lti_solve) that runs the whole
# solve when every tile's CTA fits on the GPU at once; None until the current
# version (monotone-counter grid barrier) has been captured (the previous
# version's capture: 21929472 + 8958208 bytes)
K_SOLVE_DRAM_BYTES = None


def work_model_tab(n, m, K, B, nt, wbytes):
    """FLOP and minimal DRAM bytes per time step of the tiled-scan solve with
    per-step tables (k_lti_scan), counted from the kernel for the tiles after
    the stationary point (all but a few of the tiles):
      per step: the filter offset E^T v + G y_{k+1} in phase 1 and again in
      phase 2 (2 (n^2 + n m) MAC), g_k = E (A^-1 C v + A^-1 b) (2 n^2), the
      RTS map's offset and the RTS step itself (2 n^2);
      per thread (spread over its K steps): the warp shuffle scans of the
      filter and RTS offsets with the power table (2 x 5 levels of n^2), the
      warp carries (B / 32 - 1 of n^2 per direction) and the thread's start
      values (4 n^2);
      per tile (spread over its B K steps): the tile prefix and suffix sums
      (about nt / 2 terms of n^2 each).
    Bytes: y in and x out (the per-step constants are plan-time tables of at
    most a few MB, L2-resident)."""
    L = B * K
    per_step = 2 * (n * n + n * m) + 2 * n * n + 2 * n * n
    per_thread = 2 * 5 * n * n + 2 * (B // 32 - 1) * n * n + 4 * n * n
    per_tile = 2 * (nt / 2.0) * n * n
    mac = per_step + per_thread / K + per_tile / L
    return 2 * mac, wbytes * (m + n)


# DRAM bytes (read + write) of one k_lti_scan launch on the nx=4, T=2^20
# FP32 workload from one ncu capture of the current version
# (profiles/k_lti_scan_wv4_T2p20_fp32.md): 9 427 456 B read, 0 B written (the
# states are still in L2 when the kernel ends); None once the kernel changes
K_SCAN_DRAM_BYTES = 9427456


def solve_bytes(n, m, wbytes):
    """Minimal bytes of one solve per step: y in, x out (the rest is intermediate)."""
    return wbytes * (m + n)


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    Q = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_uuid):
        self.proc = None
        self.lines = []
        try:
            cmd = ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "100"]
            if device_uuid:
                cmd += ["-i", device_uuid]
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self, t0, t1):
        rows = []
        for l in self.lines:
            p = [x.strip() for x in l.split(",")]
            if len(p) < 9:
                continue
            try:
                ts = time.mktime(time.strptime(p[0].split(".")[0], "%Y/%m/%d %H:%M:%S")) + \
                    float("0." + p[0].split(".")[1]) if "." in p[0] else 0.0
                rows.append((ts, float(p[1]), float(p[2]), p))
            except Exception:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "note": "nvidia-smi gave no samples"}
        inside = [r for r in rows if t0 - 0.15 <= r[0] <= t1 + 0.15]
        note = "samples inside the timed region"
        if not inside:
            inside = rows
            note = "timed region shorter than the sampling period: samples of warm-up + timed region"
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in inside for i in range(4) if r[3][5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": max(r[2] for r in inside),
                "reasons": reasons, "samples": len(inside), "note": note}


# ----------------------------------------------------------------------------
# oracle timing (CPU baseline and the reference arm)
# ----------------------------------------------------------------------------
def time_oracle(model, y, budget_s, min_runs=1):
    """Mean seconds per oracle solve over runs filling budget_s, the run count and the trajectory."""
    import oracle
    runs, t_tot, x = 0, 0.0, None
    while runs < min_runs or t_tot < budget_s:
        t = time.perf_counter()
        x = oracle.smooth_lti(model, y, DT)
        t_tot += time.perf_counter() - t
        runs += 1
    return t_tot / runs, runs, x


def time_oracle_batch():
    """The oracle on the 4096-trajectory batch over all host cores, one
    trajectory per thread (the C oracle releases the GIL in its ctypes calls)."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle
    from paper_2512_13319_gb300 import synth
    models, lengths, model_of, ys = synth.batched_workload()
    cores = os.cpu_count() or 1
    t = time.perf_counter()
    with ThreadPoolExecutor(max_workers=cores) as ex:
        list(ex.map(lambda j: oracle.smooth_lti(models[model_of[j]], ys[j], 0.01), range(len(lengths))))
    dt = time.perf_counter() - t
    return {"value": float(lengths.sum()) / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "all 4096 trajectories, one trajectory per thread (FP64 KF + RTS, plain C)", **host_cpu()}


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    # per-step sample sized so that warm-up + timed steps take about a minute
    model, y_full = model_and_data(1001)
    probe_T = 2 ** 14
    t_probe, _, _ = time_oracle(model, y_full[:probe_T], 0.2)
    per_step = t_probe / probe_T
    budget = 60.0 / max(1, args.steps + args.warmup)
    Ts = int(min(T_FULL, max(1024, budget / per_step)))
    y = y_full[:Ts]
    for _ in range(args.warmup):
        oracle.smooth_lti(model, y, DT)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.smooth_lti(model, y, DT)
    dt_run = (time.perf_counter() - t0) / args.steps
    value = Ts / dt_run
    sample = f"first {Ts} of the 2^20 intervals per step (FP64 KF + RTS, plain C, 1 thread)"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt_run * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "T": Ts, "nx": 4, "ny": 2, "precision": "fp64"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                         **host_cpu()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)
    return 0


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------
def ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2512_13319_gb300 import MapSmoother
    from paper_2512_13319_gb300 import build as _b

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    _b.build()

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(v):
        if world == 1:
            return v
        t = torch.tensor([v], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    prec = args.precision
    dtype = torch.float32 if prec == "fp32" else torch.float64
    wbytes = 4 if prec == "fp32" else 8
    model, y_np = model_and_data(1001 + rank)
    T = T_FULL
    y = torch.tensor(y_np, dtype=dtype, device=dev)
    x = torch.empty((T + 1, 4), dtype=dtype, device=dev)
    sm = MapSmoother(model, T, DT, precision=prec)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device=dev)

    for _ in range(max(3, args.warmup)):
        sm.solve(y, x_out=x)
    torch.cuda.synchronize(dev)

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        uuid = None
    sampler = ClockSampler(uuid)
    time.sleep(0.3)                  # let the sampler start before the timed region
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize(dev)
    t_wall0 = time.time()
    for i in range(args.steps):
        flush.zero_()
        starts[i].record(stream)
        sm.solve(y, x_out=x)
        ends[i].record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    t_wall1 = time.time()
    time.sleep(0.25)
    sampler.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    # the output of the last timed solve, kept before any other solve reuses x
    x_timed = x.clone()
    kernels_per_solve = sm.launches()          # of the timed solves
    solve_path = sm.path()
    ms_mean = max_over_ranks(sum(step_ms) / args.steps)
    ms = max_over_ranks(statistics.median(step_ms))      # median step time, max over ranks
    value = world * T / (ms * 1e-3)
    clocks = sampler.summary(t_wall0, t_wall1)

    # end to end through the host-buffer C-ABI call (H2D of y, D2H of x inside)
    y_host = torch.tensor(y_np, dtype=dtype).pin_memory()
    x_host = torch.empty((T + 1, 4), dtype=dtype).pin_memory()
    for _ in range(3):
        sm.solve_host(y_host, x_host)
    ke = max(3, min(args.steps, 50))
    barrier()
    t = time.perf_counter()
    for _ in range(ke):
        sm.solve_host(y_host, x_host)
    e2e_s = max_over_ranks((time.perf_counter() - t) / ke)
    e2e = {"value": world * T / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(y_host.numel() * wbytes),
           "d2h_bytes_per_step": int(x_host.numel() * wbytes), "ms_per_step": e2e_s * 1e3}

    # geometry of the timed path (read before the profiled solves below, which
    # run the three-kernel pipeline with its own geometry)
    K_g, B_g, nt_g = sm.geometry()
    # per-phase device times (profiled solves, L2 flushed before each; these run
    # the three-kernel pipeline, whose kernel boundaries the events mark)
    sm.profile(True)
    phases = {}
    for _ in range(10):
        flush.zero_()
        sm.solve(y, x_out=x)
        for k, v in sm.phase_times().items():
            phases.setdefault(k, []).append(v)
    sm.profile(False)
    phase_ms = {k: statistics.median(v) for k, v in phases.items()}
    K_p, B_p, nt_p = sm.geometry()             # the profiled pipeline's
    flops, byt = work_model(4, 2, K_p, B_p, nt_p, wbytes, r=2)
    peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    try:
        fma = measure_fma_peaks(dev, stream)
        alu_peak = fma["fp32"] if prec == "fp32" else fma["fp64"]
        peak_source = (f"measured on this GPU by map_fma_peak ({'FP32' if prec == 'fp32' else 'FP64'}, "
                       f"SM clock median {fma['clocks'].get('sm_mhz')} MHz during it)")
    except Exception as e:           # keep the line; fall back to unit counts
        fma = {"error": f"{type(e).__name__}: {e}"[:200]}
        fp32_nominal = SMS * FP32_LANES_PER_SM * 2 * MAX_SM_MHZ * 1e6 / 1e12
        alu_peak = fp32_nominal if prec == "fp32" else fp32_nominal / 64.0
        peak_source = "nominal unit counts (map_fma_peak failed)"
    if solve_path == 1:
        # the single launch with per-step tables: its duration is the timed
        # solve; its algorithmic work and bytes per step from work_model_tab
        flop_step, byte_step = work_model_tab(4, 2, K_g, B_g, nt_g, wbytes)
        achieved_tf = flop_step * T / (ms * 1e-3) / 1e12
        achieved_gb = byte_step * T / (ms * 1e-3) / 1e9
        fa, fh = achieved_tf / alu_peak, achieved_gb / hbm_peak
        roofline = {"bound": "alu" if fa >= fh else "hbm",
                    "achieved": achieved_tf if fa >= fh else achieved_gb,
                    "peak": alu_peak if fa >= fh else hbm_peak,
                    "unit": "TFLOP/s" if fa >= fh else "GB/s", "frac": max(fa, fh),
                    "traffic": K_SCAN_DRAM_BYTES if prec == "fp32" else None,
                    "kernel": "k_lti_scan (tiled affine scan with per-step tables: three phases, two grid barriers, one launch)",
                    "alu": {"achieved_tflops": achieved_tf, "peak_tflops": alu_peak, "frac": fa,
                            "flop_per_step": flop_step, "peak_source": peak_source},
                    "hbm": {"achieved_gbs": achieved_gb, "peak_gbs": hbm_peak, "frac": fh,
                            "bytes_per_step": byte_step, "peak_source": "MEASURED_PEAKS.json hbm_gbs"},
                    "note": "neither pipe is saturated: the solve is bound by the latency of its two "
                            "grid barriers, about 2 us each, and of the per-thread recursions"}
    elif kernels_per_solve == 1:
        # one cooperative launch runs the whole solve: its duration is the
        # timed solve, its work the three phases' work
        flop_step = sum(flops.values())
        achieved_tf = flop_step * T / (ms * 1e-3) / 1e12
        roofline = {"bound": "alu", "achieved": achieved_tf, "peak": alu_peak, "unit": "TFLOP/s",
                    "frac": achieved_tf / alu_peak,
                    "traffic": K_SOLVE_DRAM_BYTES if prec == "fp32" else None,
                    "kernel": "k_lti_solve (reduce + filter down-sweep + RTS phases, one launch)",
                    "peak_source": peak_source, "flop_per_step": flop_step}
    else:
        dom = max(("filter_reduce", "filter_down", "rts_down"), key=lambda k: phase_ms.get(k, 0.0))
        achieved_tf = flops[dom] * T / (phase_ms[dom] * 1e-3) / 1e12
        roofline = {"bound": "alu", "achieved": achieved_tf, "peak": alu_peak, "unit": "TFLOP/s",
                    "frac": achieved_tf / alu_peak,
                    "traffic": K_FILTER_DOWN_DRAM_BYTES if (dom == "filter_down" and prec == "fp32") else None,
                    "kernel": dom, "peak_source": peak_source, "flop_per_step": flops[dom]}
    per_phase = {k: {"ms": phase_ms[k],
                     "tflops": (flops[k] * T / (phase_ms[k] * 1e-3) / 1e12) if k in flops else None,
                     "gbs_min_bytes": (byt[k] * T / (phase_ms[k] * 1e-3) / 1e9) if k in byt else None}
                 for k in phase_ms}
    hbm = {"solve_min_bytes_per_step": solve_bytes(4, 2, wbytes),
           "achieved_gbs": solve_bytes(4, 2, wbytes) * T / (ms * 1e-3) / 1e9, "peak_gbs": hbm_peak,
           "note": "y in + x out over the whole solve; intermediates excluded"}
    hbm["frac"] = hbm["achieved_gbs"] / hbm_peak
    fb, sing, timeouts = sm.stats()
    # kernels of one timed solve, as the library reports them (1 for the single
    # cooperative launch; else reduce, group totals, filter down-sweep, RTS pass)
    launches_per_solve = kernels_per_solve

    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if prec == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "T": T, "nx": 4, "ny": 2, "precision": prec,
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": "flushed before every timed step (256 MiB write)",
                   "steps_per_thread": K_g, "threads_per_tile": B_g, "tiles": nt_g},
        "ms_per_step_mean": ms_mean,
        "clocks": clocks, "e2e": e2e, "gpu_launches": launches_per_solve * args.steps, "roofline": roofline,
        "phases": per_phase, "hbm": hbm, "fp64_recomputes": fb, "singular_pivots": sing, "copy_wait_timeouts": timeouts,
        "fma_peaks_tflops": fma,
    }
    sm.close()

    if rank == 0 and world == 1 and not args.no_extras:
        # FP64 path on the same workload
        sm64 = MapSmoother(model, T, DT, precision="fp64")
        y64 = y.double()
        x64 = torch.empty((T + 1, 4), dtype=torch.float64, device=dev)
        for _ in range(2):
            sm64.solve(y64, x_out=x64)
        evs = []
        for _ in range(5):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sm64.solve(y64, x_out=x64)
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize(dev)
        ms64 = statistics.median(a.elapsed_time(b) for a, b in evs)
        result["fp64"] = {"value": T / (ms64 * 1e-3), "unit": UNIT, "ms_per_step": ms64}
        sm64.close()
        # sequential GPU baseline (one thread, same recursions), if built
        seq = sequential_gpu(model, y, dtype, dev, flush, stream)
        if seq:
            result["sequential_gpu"] = seq
            result["speedup_vs_sequential_gpu"] = value / seq["value"]
        result["extras"], checks = extras(dev, flush, stream)
    else:
        checks = []
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        t_run, runs, x_ref = time_oracle(model, y_np, 10.0)
        result["cpu_baseline"] = {"value": T / t_run, "unit": UNIT, "cores": 1, "kind": "oracle",
                                  "sample": f"the full T=2^20 workload, {runs} runs (FP64 KF + RTS, plain C)",
                                  **host_cpu()}
        # error of the last timed solve's own output against the oracle
        x_gpu = x_timed.double().cpu().numpy()
        result["rel_err_vs_oracle"] = float(np.linalg.norm(x_gpu - x_ref) / np.linalg.norm(x_ref))
        result["max_abs_err_rel_to_max_vs_oracle"] = float(np.abs(x_gpu - x_ref).max() / np.abs(x_ref).max())
        if checks and "extras" in result:
            oracle_checks(result["extras"], checks)
            b = result["extras"].get("batched")
            if isinstance(b, dict) and "error" not in b:
                b["cpu_all_cores"] = time_oracle_batch()
    elif "extras" in result:
        for name, key, *_ in checks:
            if isinstance(result["extras"].get(name), dict) and "error" not in result["extras"][name]:
                result["extras"][name][key] = "not checked (CPU-baseline leg skipped)"
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def timed(fn, flush, stream, dev, reps=3):
    """Median device time (ms) of fn() with the L2 flushed before each call."""
    import torch
    fn()
    times = []
    for _ in range(reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize(dev)
        times.append(a.elapsed_time(b))
    return statistics.median(times)


def measure_fma_peaks(dev, stream):
    """FP32 and FP64 FMA throughput of this GPU (TFLOP/s), measured with the
    library's map_fma_peak kernels (8 CTAs x 256 threads per SM, 8 independent
    chains per thread), best of 5 launches of about 50 ms each, with the SM
    clock sampled during them."""
    import torch

    from paper_2512_13319_gb300 import _binding as B
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    sampler = ClockSampler(uuid)
    time.sleep(0.3)
    t0 = time.time()
    out = {}
    st = stream.cuda_stream
    for name, kind, iters in (("fp32_ffma", B.FMA_FP32, 50_000), ("fp32_ffma2", B.FMA_FP32X2, 25_000),
                              ("fp64_dfma", B.FMA_FP64, 750)):
        B.map_fma_peak(kind, max(1, iters // 10), st)       # warm-up
        best = 0.0
        for _ in range(5):
            flop, ms = B.map_fma_peak(kind, iters, st)
            best = max(best, flop / (ms * 1e-3) / 1e12)
        out[name] = best
    t1 = time.time()
    time.sleep(0.25)
    sampler.stop()
    out["clocks"] = sampler.summary(t0, t1)
    out["fp32"] = max(out["fp32_ffma"], out["fp32_ffma2"])
    out["fp64"] = out["fp64_dfma"]
    out["how"] = ("map_fma_peak: 8 CTAs x 256 threads per SM, 8 independent FMA chains per thread, "
                  "best of 5 launches of ~50 ms; fp32 = max(scalar FFMA, paired FFMA2)")
    return out


def host_cpu():
    """CPU model and logical core count of this host (for the CPU baselines)."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k = line.split(":")[0].strip().lower()
                if k in ("model name", "cpu model", "hardware"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if not model:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    import platform
    return {"cpu_model": model or platform.processor() or platform.machine(), "nproc": os.cpu_count()}


def rel_err(a, b):
    import numpy as np
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def hbm_peak_gbs():
    peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
    return peaks.get("hbm_gbs", 6800.0)


def extras(dev, flush, stream):
    """The other workloads of the path, timed on the GPU.  Returns the results
    and the checks that the CPU-baseline leg resolves with the oracle (extra,
    result key, oracle function, its arguments, the GPU result); no oracle call
    happens here."""
    import numpy as np
    import torch

    from paper_2512_13319_gb300 import MapSmoother, synth
    out = {}
    checks = []

    def guard(name, fn):
        try:
            out[name] = fn()
        except Exception as e:          # report, do not lose the main line
            out[name] = {"error": f"{type(e).__name__}: {e}"[:300]}

    def ou8():
        model = synth.ou_model(8, 4, seed=1001)
        _, y = synth.simulate(model, T_FULL, DT, seed=1011, substeps=1)
        sm = MapSmoother(model, T_FULL, DT, precision="fp32")
        yt = torch.tensor(y, dtype=torch.float32, device=dev)
        x = torch.empty((T_FULL + 1, 8), dtype=torch.float32, device=dev)
        ms = timed(lambda: sm.solve(yt, x_out=x), flush, stream, dev)
        checks.append(("ou_nx8", "rel_err_vs_oracle", "smooth_lti", (model, y, DT), x.cpu().numpy()))
        sm.close()
        return {"workload": "OU nx=8 ny=4, T=2^20, dt=1e-3, FP32, RTS", "ms": ms,
                "value": T_FULL / (ms * 1e-3), "unit": UNIT}

    def two_filter():
        model, y = model_and_data(1001)
        sm = MapSmoother(model, T_FULL, DT, precision="fp32", smoother="two_filter")
        yt = torch.tensor(y, dtype=torch.float32, device=dev)
        x = torch.empty((T_FULL + 1, 4), dtype=torch.float32, device=dev)
        ms = timed(lambda: sm.solve(yt, x_out=x), flush, stream, dev)
        checks.append(("two_filter", "rel_err_vs_oracle", "smooth_lti", (model, y, DT), x.cpu().numpy()))
        sm.close()
        return {"workload": "Wiener velocity nx=4, T=2^20, FP32, two-filter smoother", "ms": ms,
                "value": T_FULL / (ms * 1e-3), "unit": UNIT}

    def coord_turn():
        model = synth.coordinated_turn()
        T, iters = 2 ** 16, 10
        _, y = synth.simulate(model, T, DT, seed=1002)
        x0 = np.tile(model.m0, (T + 1, 1))
        sm = MapSmoother(model, T, DT, precision="fp32", gn_iters=iters)
        yt = torch.tensor(y, dtype=torch.float32, device=dev)
        xi = torch.tensor(x0, dtype=torch.float32, device=dev)
        x = torch.empty_like(xi)
        ms = timed(lambda: sm.solve(yt, x_out=x, x_init=xi), flush, stream, dev)
        checks.append(("coordinated_turn", "rel_err_vs_oracle", "gauss_newton", (model, y, DT, x0, iters),
                       x.cpu().numpy()))
        seq = torch.empty_like(xi)
        ms_seq = timed(lambda: sm.solve_sequential(yt, x_out=seq, x_init=xi), flush, stream, dev, reps=1)
        sm.close()
        return {"workload": "coordinated turn nx=5 ny=2, T=2^16, dt=1e-3, 10 Gauss-Newton iterations, FP32",
                "ms": ms, "value": T * iters / (ms * 1e-3), "unit": "time-steps x iterations/s",
                "sequential_gpu_ms": ms_seq,
                "speedup_vs_sequential_gpu": ms_seq / ms}

    def coord_turn_expm():
        # Gauss-Newton with each step's linearised drift discretised exactly
        model = synth.coordinated_turn()
        T, iters = 2 ** 16, 10
        _, y = synth.simulate(model, T, DT, seed=1002)
        x0 = np.tile(model.m0, (T + 1, 1))
        sm = MapSmoother(model, T, DT, precision="fp32", gn_iters=iters, discretisation="expm")
        yt = torch.tensor(y, dtype=torch.float32, device=dev)
        xi = torch.tensor(x0, dtype=torch.float32, device=dev)
        x = torch.empty_like(xi)
        ms = timed(lambda: sm.solve(yt, x_out=x, x_init=xi), flush, stream, dev)
        checks.append(("coordinated_turn_expm", "rel_err_vs_oracle", "gauss_newton",
                       (model, y, DT, x0, iters, 1), x.cpu().numpy()))     # mode 1: exact discretisation
        sm.close()
        return {"workload": "coordinated turn nx=5 ny=2, T=2^16, dt=1e-3, 10 Gauss-Newton iterations, each step's "
                            "linearised drift discretised exactly, FP32", "ms": ms,
                "value": T * iters / (ms * 1e-3), "unit": "time-steps x iterations/s"}

    def batched():
        from paper_2512_13319_gb300.batch import MapBatch
        models, lengths, model_of, ys = synth.batched_workload()
        mb = MapBatch(models, lengths, model_of, [0.01] * len(models), precision="fp32")
        yd = mb.pack_observations(ys)
        xd = mb.empty_outputs()
        mb.solve(yd, xd)                 # autotune + graph capture
        ms = timed(lambda: mb.solve(yd, xd), flush, stream, dev)
        xs = mb.unpack_states(xd)
        rng = np.random.default_rng(0)
        for j in rng.choice(len(lengths), size=20, replace=False):
            checks.append(("batched", "max_rel_err_vs_oracle_20_sampled", "smooth_lti",
                           (models[model_of[j]], ys[j], 0.01), xs[j]))
        KB, B = mb.tuning(0)
        persistent = mb.persistent()
        mb.close()
        steps = int(lengths.sum())
        # bytes the persistent kernel must move: y read twice (forward and
        # backward sweeps) and x written once, per step of each model
        nx_of = np.array([models[m].nx for m in model_of])
        ny_of = np.array([models[m].ny for m in model_of])
        min_bytes = float(np.sum(lengths * (2 * ny_of + nx_of) * 4 + nx_of * 4))
        return {"workload": "4096 Wiener-velocity trajectories, nx in {2,4,6}, lengths log-uniform 256..65536, "
                            "dt=0.01, FP32, one persistent launch in a CUDA graph", "steps": steps, "ms": ms,
                "value": steps / (ms * 1e-3), "unit": UNIT, "persistent_kernel": persistent,
                "steps_per_thread": KB, "threads_per_cta": B,
                "hbm": {"bytes": min_bytes, "gbs": min_bytes / (ms * 1e-3) / 1e9,
                        "frac": min_bytes / (ms * 1e-3) / 1e9 / hbm_peak_gbs(),
                        "note": "y read in both sweeps + x written, per step (model-dependent sizes)"}}

    def gradient():
        T = 2 ** 18
        model = synth.ou_model(4, 2, seed=51)
        _, y = synth.simulate(model, T, DT, seed=1004, substeps=1)
        sm = MapSmoother(model, T, DT, precision="fp32")
        yt = torch.tensor(y, dtype=torch.float32, device=dev)
        x = sm.solve(yt)
        box = {}

        def step():
            sm.solve(yt, x_out=x)
            box["g"] = sm.grad(yt, x)
        ms = timed(step, flush, stream, dev)
        checks.append(("gradient", "rel_err_vs_fp64_oracle_gradient", "grad_lti", (model, y, DT),
                       np.asarray(box["g"])))
        sm.close()
        return {"workload": "MAP-cost gradient w.r.t. (F 4x4, log q, log r), OU nx=4, T=2^18, FP32 "
                            "(solve + adjoint solve + contraction)", "ms": ms}

    def parameter_update():
        # a learning step changes theta: set-up and plan-time constants again
        # (discretisation, folds, tile tables, products), then one solve
        T = 2 ** 18
        model = synth.ou_model(4, 2, seed=51)
        _, y = synth.simulate(model, T, DT, seed=1004, substeps=1)
        sm = MapSmoother(model, T, DT, precision="fp32")
        yt = torch.tensor(y, dtype=torch.float32, device=dev)
        x = sm.solve(yt)

        def step():
            sm.update(F=model.F, log_q=0.0, log_r=0.0)
            sm.solve(yt, x_out=x)
        ms = timed(step, flush, stream, dev)
        solve_ms = timed(lambda: sm.solve(yt, x_out=x), flush, stream, dev)
        sm.close()
        return {"workload": "parameter update + solve, OU nx=4, T=2^18, FP32", "ms": ms,
                "solve_only_ms": solve_ms}

    def block_dense():
        # Section 5.1 block elements (10 Euler substeps per interval) and the
        # dense output at every substep
        model = synth.ou_model(4, 2, seed=1001)
        nsub = 10
        _, y = synth.simulate(model, T_FULL, DT, seed=1012, substeps=1)
        sm = MapSmoother(model, T_FULL, DT, precision="fp32", discretisation="block", substeps=nsub)
        yt = torch.tensor(y, dtype=torch.float32, device=dev)
        x = torch.empty((T_FULL + 1, 4), dtype=torch.float32, device=dev)
        ms = timed(lambda: sm.solve(yt, x_out=x), flush, stream, dev)
        x, f, _ = sm.solve(yt, filt=True)
        xd = torch.empty((T_FULL * nsub + 1, 4), dtype=torch.float32, device=dev)
        ms_dense = timed(lambda: sm.dense(yt, x, f, out=xd), flush, stream, dev)
        checks.append(("block_elements", "rel_err_vs_oracle", "smooth_block", (model, y, DT, nsub),
                       x.cpu().numpy()))
        checks.append(("block_elements", "dense_rel_err_vs_oracle", "dense_block", (model, y, DT, nsub),
                       xd.cpu().numpy()))
        sm.close()
        return {"workload": "OU nx=4 ny=2, T=2^20, dt=1e-3, block elements of 10 Euler substeps, FP32, RTS; "
                            "dense output at all 10 T + 1 substep times", "ms": ms,
                "value": T_FULL / (ms * 1e-3), "unit": UNIT, "dense_ms": ms_dense}

    def exact():
        model = synth.ou_model(4, 2, seed=1001)
        _, y = synth.simulate(model, T_FULL, DT, seed=1013, substeps=1)
        sm = MapSmoother(model, T_FULL, DT, precision="fp32", discretisation="exact")
        yt = torch.tensor(y, dtype=torch.float32, device=dev)
        x = torch.empty((T_FULL + 1, 4), dtype=torch.float32, device=dev)
        ms = timed(lambda: sm.solve(yt, x_out=x), flush, stream, dev)
        checks.append(("exact_elements", "rel_err_vs_oracle", "smooth_exact", (model, y, DT), x.cpu().numpy()))
        sm.close()
        return {"workload": "OU nx=4 ny=2, T=2^20, dt=1e-3, exact elements (Eq. 37 solved over each "
                            "interval), FP32, RTS", "ms": ms, "value": T_FULL / (ms * 1e-3), "unit": UNIT}

    for name, fn in (("ou_nx8", ou8), ("two_filter", two_filter), ("coordinated_turn", coord_turn),
                     ("coordinated_turn_expm", coord_turn_expm),
                     ("batched", batched), ("gradient", gradient), ("parameter_update", parameter_update),
                     ("block_elements", block_dense), ("exact_elements", exact)):
        guard(name, fn)
    return out, checks


def oracle_checks(out, checks):
    """CPU-baseline leg: each extra's GPU result against the FP64 oracle on the
    same inputs (relative Frobenius error; several checks under one key keep the
    largest).  A check that raises records its error text under
    ``<key>_errors``; the numeric key keeps the largest error of the others."""
    import numpy as np

    import oracle
    for name, key, fn, args, got in checks:
        if not isinstance(out.get(name), dict) or "error" in out[name]:
            continue
        try:
            ref = getattr(oracle, fn)(*args)
            if isinstance(ref, tuple):
                ref = ref[0]
            err = rel_err(got, ref)
            prev = out[name].get(key)
            out[name][key] = err if not isinstance(prev, float) else max(prev, err)
            if fn == "grad_lti":          # per-block errors of (F, log q, log r)
                n2 = len(ref) - 2
                out[name]["rel_err_F_block"] = rel_err(got[:n2], ref[:n2])
                out[name]["rel_err_log_q"] = abs(got[n2] - ref[n2]) / abs(ref[n2])
                out[name]["rel_err_log_r"] = abs(got[n2 + 1] - ref[n2 + 1]) / abs(ref[n2 + 1])
                out[name]["max_abs_err_F_rel_to_max_F"] = float(np.abs(got[:n2] - ref[:n2]).max()
                                                                / np.abs(ref[:n2]).max())
            else:
                mx = float(np.abs(np.asarray(got) - ref).max() / np.abs(ref).max())
                pk = "max_abs_err_rel_to_max"
                out[name][pk] = mx if not isinstance(out[name].get(pk), float) else max(out[name][pk], mx)
        except Exception as e:          # report, do not lose the main line
            out[name].setdefault(key + "_errors", []).append(f"{type(e).__name__}: {e}"[:200])


def sequential_gpu(model, y, dtype, dev, flush, stream):
    try:
        from paper_2512_13319_gb300 import sequential
    except Exception:
        return None
    return sequential.time_sequential(model, y, DT, dtype, dev, flush, stream)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return reference_arm(args)
    return ours(args)


if __name__ == "__main__":
    sys.exit(main())
