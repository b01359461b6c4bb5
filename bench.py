#!/usr/bin/env python
"""Benchmark of the NLINV hot path on one GB300: the real-time radial series of Sec. 3.2.

Workload: 384 x 384 grid (192 x 192 image, 2x oversampled), 10 virtual coils, 13 radial spokes per frame rotated by
k * 2 pi / 65 from frame to frame, 7 Gauss-Newton steps x 30 CG iterations per frame, each frame initialised from
and regularised toward the previous one.  One step = one frame reconstruction (every row of the hot path).
Inputs are synthetic (seeded phantom, Gaussian coil maps, radial masks, 30 dB noise) and resident in HBM before
the timed region; L2 is flushed before every frame.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the CPU oracle instead, on bounded samples.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "NLINV frames/s and p99 frame latency (384^2, 10 coils); operator % HBM roofline"
WORKLOAD = "realtime_384"
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=195)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--batch-profile", action="store_true",
                    help="with --workload batch64: build the batch and run one reconstruction, untimed (for ncu)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the compiled launch shapes (profiling runs: the tuner replays ~30k launches)")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the 64-frame uneven batch (batched vs plain per-frame) after the series")
    ap.add_argument("--no-precision", action="store_true",
                    help="skip the 512x512, 16-coil precision comparison (FP32 vs tensor-core DFT stages)")
    ap.add_argument("--workload", default=WORKLOAD, choices=[WORKLOAD, "batch64"],
                    help="realtime_384 (default): the real-time series; batch64: 64 independent frames of uneven "
                         "grid side and coil count, batched against plain per-frame reconstruction")
    ap.add_argument("--write-traffic", metavar="NCU_REP",
                    help="read the DRAM bytes of the CG kernels from an ncu report of paper_1301_1215_gb300.profile_cg "
                         "and write profiles/traffic.json (no GPU needed)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def csrc_digest() -> str:
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1301_1215_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".cuh")):
            with open(os.path.join(d, f), "rb") as fh:
                h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


# ----------------------------------------------------------------------------------------------- clocks ----
class ClockSampler:
    """nvidia-smi clock and throttle samples every 200 ms while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------------------------- workload ----
def build_series(torch, ctx, W, frames, dev):
    """Seeded truth (static object), per-frame radial masks and noisy data y_k = P FFT(M rho c_j) + noise,
    generated on the device with the library's own simulation kernel."""
    import numpy as np
    from paper_1301_1215_gb300 import synth
    fr = synth.make_frame(W.n, W.ncoils, W.spokes, seed=W.seed)
    rho = torch.from_numpy(fr.rho.astype(np.complex64)).to(dev)
    coils = torch.from_numpy(fr.coils.astype(np.complex64)).to(dev)
    masks = torch.stack([torch.from_numpy(synth.radial_mask(W.n, W.spokes, synth.frame_rotation(k, W.spokes)))
                         for k in range(frames)]).to(dev)
    ys = torch.empty((frames, W.ncoils, W.n, W.n), dtype=torch.complex64, device=dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(W.seed)
    sigma = None
    for k in range(frames):
        ctx.simulate(rho, coils, masks[k], out=ys[k])
        if sigma is None:
            npts = float(masks[k].sum().item()) * W.ncoils
            power = float((ys[k].abs() ** 2).sum().item()) / npts
            sigma = synth.noise_sigma(power, W.snr_db)
        noise = torch.randn((W.ncoils, W.n, W.n, 2), generator=gen, device=dev) * (sigma * 0.5 ** 0.5)
        ys[k] += torch.view_as_complex(noise) * masks[k]
    torch.cuda.synchronize()
    return ys, masks


def max_over_ranks(value: float, device) -> float:
    """Largest value over the ranks of the default process group (the value itself on one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(steps_per_rank: int, world: int, slowest_ms: float) -> float:
    """Whole-job frames/s of `world` independent replicas that each reconstructed steps_per_rank frames, the
    slowest taking slowest_ms (replicas only: the frames of different ranks never exchange data)."""
    return world * steps_per_rank / (slowest_ms / 1e3)


def cg_bytes(n: int, J: int, fov: int):
    """Algorithmic bytes per launch of the kernels of one CG iteration: every input read once and every output
    written once (U = one complex64 plane, compact Omega columns Wc = 2 fov)."""
    U = n * n * 8
    h = (2 * fov) / n                 # fraction of a plane kept as Omega columns
    q = h * h                         # fraction kept as Omega
    mask = n * n
    return {
        "row p-update/W^-1": J * U * (3 + h),                          # r_c, p_c in; p_c, T out
        "col W^-1/C/FFT": J * U * (h + q + h) + 3 * q * U,             # T, c in; T out; rho, r_rho, p_rho on Omega
        "row PSF": J * U * 2 * h + mask,
        "col FFT^-1/C^H/FFT": J * U * (h + q + h + q) + q * U,         # T, c in; T, channel products out; rho
        "row W^-H+alpha p": J * U * (h + q) + 2 * J * U + 4 * U,       # T, products, p in; q out; rho: r, p in, p, q out
        "cg step": 6 * (1 + J) * U,                                    # p, q, r, dx in; dx, r out
    }


def compulsory_bytes(n: int, J: int) -> int:
    """Compulsory bytes of one CG iteration: the normal operator reads p, c, rho and the mask and writes q
    ((3J + 3) planes + n^2 bytes), the CG update reads x, r, p, q and writes x, r, p (7 (1 + J) planes): every
    array touched once, whatever the kernel design."""
    U = n * n * 8
    return (10 * J + 10) * U + n * n


def run_ours(args, rank, world, local):
    import numpy as np
    import torch
    from paper_1301_1215_gb300 import synth
    from paper_1301_1215_gb300.build import build
    from paper_1301_1215_gb300.nlinv import Nlinv

    build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    W = synth.WORKLOADS[WORKLOAD]
    K, Wm = args.steps, args.warmup
    frames = K + Wm
    ctx = Nlinv(W.n, W.ncoils, newton_steps=W.newton_steps, cg_iters=W.cg_iters, alpha0=W.alpha0,
                alpha_q=W.alpha_q, sobolev_a=W.sobolev_a, sobolev_l=W.sobolev_l, use_graph=True, device=dev)
    ys, masks = build_series(torch, ctx, W, frames, dev)
    if args.no_autotune:
        tuned = {"vec_blocks_per_sm": None, "pdl": None, "split_n1": None, "col_strip": None,
                 "row_blocks_per_sm": None, "candidates": "not run (--no-autotune): compiled defaults"}
    else:
        tuned = ctx.autotune(ys[0], masks[0], reps=3)   # launch shapes from timed whole-frame graph replays
    l2 = torch.cuda.get_device_properties(dev).L2_cache_size
    flush = torch.empty(max(2 * l2, 256 << 20), dtype=torch.uint8, device=dev)
    x = torch.zeros((1 + W.ncoils, W.n, W.n), dtype=torch.complex64, device=dev)
    x[0] = 1.0

    for k in range(Wm):
        ctx.reconstruct_inplace(ys[k], masks[k], x)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.synchronize()
    launches = 0
    for i in range(K):
        k = Wm + i
        flush.zero_()
        ctx.stream.wait_stream(torch.cuda.current_stream(dev))
        starts[i].record(ctx.stream)
        ctx.reconstruct_inplace(ys[k], masks[k], x)
        ends[i].record(ctx.stream)
        launches += ctx.last_launch_count
    torch.cuda.synchronize()
    clk = clocks.stop()
    frame_ms = sorted(s.elapsed_time(e) for s, e in zip(starts, ends))
    total_ms = sum(frame_ms)
    total_ms = max_over_ranks(total_ms, dev)
    value = replica_throughput(K, world, total_ms)
    p50 = frame_ms[len(frame_ms) // 2]
    p99 = frame_ms[min(len(frame_ms) - 1, int(round(0.99 * (len(frame_ms) - 1))))]
    finite = bool(torch.isfinite(torch.view_as_real(x)).all().item())

    # per-kernel CUDA-event durations of the CG iteration on the same state (the roofline's dominant kernel)
    prof = ctx.profile_cg(reps=20)
    algo = cg_bytes(W.n, W.ncoils, W.fov)
    top = max(prof, key=prof.get)
    hbm, src = peaks()
    achieved = algo[top] / (prof[top] * 1e-3) / 1e9
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tpath):
        with open(tpath) as f:
            tj = json.load(f)
        if tj.get("csrc_digest") == csrc_digest() and top in tj.get("kernels", {}):
            traffic = tj["kernels"][top]
    kernels = {k: {"ms": round(v, 5), "algo_bytes": int(algo[k]),
                   "gbs": round(algo[k] / (v * 1e-3) / 1e9, 1)} for k, v in prof.items()}
    # the same iteration on the compulsory accounting (every array touched once): bytes / in-graph iteration time
    # (the six steady-state kernel durations add up to it), and bytes of all CG iterations / whole frame time
    t_iter = sum(prof.values()) * 1e-3
    comp = compulsory_bytes(W.n, W.ncoils)
    comp_iter_gbs = comp / t_iter / 1e9
    comp_frame_gbs = comp * W.newton_steps * W.cg_iters / (total_ms / K * 1e-3) / 1e9

    # end to end through the C interface with host buffers: pinned y and mask in, x in and out every frame
    e2e = None
    e2e_stops = []
    if not args.no_e2e:
        R = min(8, frames)
        yh = [ys[k].cpu().pin_memory() for k in range(R)]
        mh = [masks[k].cpu().pin_memory() for k in range(R)]
        xh = x.cpu().pin_memory()
        ctx.reconstruct_inplace(yh[0], mh[0], xh)
        tot = 0.0
        dev_ms = 0.0
        for i in range(K):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0 = time.perf_counter()
            e0.record(ctx.stream)
            ctx.reconstruct_inplace(yh[i % R], mh[i % R], xh)   # returns after the copy back to host memory
            tot += time.perf_counter() - t0
            e1.record(ctx.stream)
            e1.synchronize()
            dev_ms += e0.elapsed_time(e1)
            e2e_stops.append(ctx.cg_stops())
        bi = yh[0].numel() * 8 + mh[0].numel() + xh.numel() * 8
        e2e = {"value": round(world * K / tot, 3), "unit": "frames/s", "h2d_bytes_per_step": int(bi),
               "d2h_bytes_per_step": int(xh.numel() * 8), "wall_ms_per_frame": round(tot / K * 1e3, 4),
               "stream_ms_per_frame": round(dev_ms / K, 4),
               "note": "wall: host clock around the call (copies in, graph, copy out, wait); stream: CUDA events "
                       "around the same call on the context stream"}

    # the gridding of one frame's radial samples onto the grid (nlinv_grid, the pre-processing of Sec. 3.1)
    from paper_1301_1215_gb300.nlinv import Gridder
    ang = [np.pi * s_ / W.spokes + synth.frame_rotation(0, W.spokes) for s_ in range(W.spokes)]
    with Gridder(W.n, [(np.cos(a), np.sin(a)) for a in ang], device=dev) as gr:
        smp = torch.randn((W.ncoils, W.spokes, 2 * W.n), dtype=torch.complex64, device=dev)
        for _ in range(3):
            gr.grid(smp)
        torch.cuda.synchronize()
        gs, ge = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        gs.record(gr.stream)
        for _ in range(100):
            gr.grid(smp)
        ge.record(gr.stream)
        torch.cuda.synchronize()
        grid_us = gs.elapsed_time(ge) / 100 * 1e3
    gbytes = smp.numel() * 8 + W.ncoils * W.n * W.n * 8 + W.n * W.n
    gridding = {"workload": f"{W.spokes} spokes x {2 * W.n} samples x {W.ncoils} coils onto {W.n}^2",
                "us_per_frame": round(grid_us, 2), "algo_bytes": int(gbytes),
                "gbs": round(gbytes / (grid_us * 1e-6) / 1e9, 1)}

    # CG iterations a frame executes: a solve that reaches the FP32 rounding floor (|r| <= 2^-24 |b|) stops there,
    # as the oracle's does; the series' own stops, read after each end-to-end frame
    if e2e_stops:
        runs = [sum(W.cg_iters if st < 0 else st + 1 for st in f) for f in e2e_stops]
        cg_exec = {"mean_per_frame": round(sum(runs) / len(runs), 2), "max_per_frame": max(runs),
                   "scheduled_per_frame": W.newton_steps * W.cg_iters, "last_frame_stops": e2e_stops[-1],
                   "rule": "a CG solve stops at |r| <= 2^-24 |b|, Re<p,Ap> <= 0 or a non-finite value (the oracle "
                           "applies the same rule); the stopped solve's remaining launches return at once"}
    else:
        cg_exec = None
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "frames/s", "n_gpus": world, "steps": K,
        "warmup": Wm, "ms_per_step": round(total_ms / K, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c64 (f32 complex; f64 CG scalars)", "data": "synthetic",
        "p50_ms": round(p50, 4), "p99_ms": round(p99, 4),
        "config": {"workload": "real-time radial series: 384x384 grid (192x192 image), 10 coils, 13 spokes/frame "
                               "rotated k*2pi/65, 7 Newton x 30 CG, previous frame as start and reference",
                   "n": W.n, "coils": W.ncoils, "spokes": W.spokes, "newton_steps": W.newton_steps,
                   "cg_iters": W.cg_iters, "cg_iterations_executed": cg_exec, "frames_timed": K,
                   "graph": "one CUDA graph per frame",
                   "launch_shapes": {"split_n1": tuned["split_n1"], "col_strip": tuned["col_strip"],
                                     "row_blocks_per_sm": tuned["row_blocks_per_sm"],
                                     "vec_blocks_per_sm": tuned["vec_blocks_per_sm"], "pdl": tuned["pdl"],
                                     "chosen_by": "nlinv_autotune (whole-frame graph replays, one dimension per "
                                                  "stage: split, column strip, row blocks/SM, vector blocks x PDL)",
                                     "candidates": tuned["candidates"]},
                   "l2": "flushed before every frame (the frame's ~110 MB working set then stays on chip)",
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "roofline": {"bound": "hbm", "kernel": top, "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                     "frac": round(achieved / hbm, 4), "peak_source": src, "traffic": traffic,
                     "algo_bytes_per_launch": int(algo[top]), "kernels": kernels,
                     "frac_compulsory": round(comp_iter_gbs / hbm, 4),
                     "compulsory": {"bytes_per_cg_iter": int(comp), "iter_ms": round(t_iter * 1e3, 5),
                                    "gbs": round(comp_iter_gbs, 1),
                                    "frame_gbs": round(comp_frame_gbs, 1),
                                    "frame_frac": round(comp_frame_gbs / hbm, 4),
                                    "note": "(10J+10) planes + n^2 bytes per CG iteration; iter_ms = the six "
                                            "steady-state kernel durations; frame_* = all CG iterations' bytes / "
                                            "whole frame time (includes the non-CG passes)"},
                     "l2_resident": "the 384^2 frame's ~110 MB working set stays in the 126 MB L2 between passes: "
                                    "DRAM traffic ('traffic') is below the algorithmic bytes; the HBM-bound case "
                                    "is the 'batch64' key"},
        "e2e": e2e, "gpu_launches": int(launches), "clocks": clk, "finite": finite, "gridding": gridding,
    }
    if cg_exec is not None:       # bytes of the CG iterations a frame really executes / frame time
        fg = comp * cg_exec["mean_per_frame"] / (total_ms / K * 1e-3) / 1e9
        line["roofline"]["compulsory"]["frame_gbs"] = round(fg, 1)
        line["roofline"]["compulsory"]["frame_frac"] = round(fg / hbm, 4)
        line["roofline"]["compulsory"]["note"] = line["roofline"]["compulsory"]["note"].replace(
            "all CG iterations' bytes", "the executed CG iterations' bytes")
    ctx.close()
    if world > 1:       # replicas: the series alone; the single-GPU legs below would only hold every GPU longer
        line["extras"] = "batch64, precision_512 and cpu_baseline are measured at N = 1 only"
        return line
    if not args.no_batch:
        line["batch64"] = batch_compare(torch, dev, K=3, Wm=1)
    if not args.no_precision:
        line["precision_512"] = precision_compare(torch, dev)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(W)
    return line


# ------------------------------------------------------------------------------------------ CPU oracle ----
def _oracle_problem(W):
    import numpy as np
    import oracle.nlinv_oracle as O
    from paper_1301_1215_gb300 import synth
    s = O.Setup(W.n, W.ncoils, W.fov, W.sobolev_a, W.sobolev_l)
    fr = synth.make_frame(W.n, W.ncoils, W.spokes, seed=W.seed)
    y0 = O.simulate(s, fr.mask, fr.rho, fr.coils)
    power = float(np.sum(np.abs(y0) ** 2) / (fr.mask.sum() * W.ncoils))
    y = y0 + fr.mask * synth.noise_sigma(power, W.snr_db) * fr.noise
    return O, s, fr, y, synth.initial_guess(W.n, W.ncoils)


def cpu_baseline(W):
    """The oracle, as it stands, on one bounded sample: frame 0 of the series, a whole reconstruction (7 Newton
    steps, CG to the rounding floor or 30 iterations), plus one normal-operator application and the small
    64 x 64 single frame."""
    O, s, fr, y, x0 = _oracle_problem(W)
    c0 = cpu_seconds()
    t0 = time.perf_counter()
    stops = []
    O.irgnm(s, fr.mask, y, x0, None, W.newton_steps, W.cg_iters, cg_stops=stops)
    dt = time.perf_counter() - t0
    cores = max(1, round((cpu_seconds() - c0) / dt))
    iters = sum(W.cg_iters if st < 0 else st + 1 for st in stops)
    # one application of the normal operator (DF^H DF + alpha) on the same problem, coil maps given
    c = O.coils(s, x0)
    t1 = time.perf_counter()
    O.normal(s, fr.mask, x0, x0, W.alpha0, c)
    normal_ms = (time.perf_counter() - t1) * 1e3
    # the small single-frame case (64 x 64 grid, 4 coils, 16 spokes, 7 Newton x 30 CG), a whole reconstruction
    from paper_1301_1215_gb300 import synth
    W1 = synth.WORKLOADS["single_64"]
    O1, s1, fr1, y1, x01 = _oracle_problem(W1)
    t2 = time.perf_counter()
    O1.irgnm(s1, fr1.mask, y1, x01, None, W1.newton_steps, W1.cg_iters)
    small_s = time.perf_counter() - t2
    return {"value": round(1.0 / dt, 6), "unit": "frames/s", "cores": cores, "kind": "oracle",
            "host_cores": os.cpu_count(), "s_per_frame": round(dt, 2), "cg_iterations": iters, "cg_stops": stops,
            "normal_op_ms": round(normal_ms, 1), "single_64_s_per_frame": round(small_s, 3),
            "sample": f"frame 0 of the series, one whole reconstruction (numpy complex128, {W.newton_steps} "
                      f"Newton steps, {iters} CG iterations to the rounding floor or {W.cg_iters}), {dt:.1f} s; "
                      f"normal_op_ms: one (DF^H DF + alpha) application on the same frame; single_64_s_per_frame: "
                      f"one whole reconstruction of the 64x64, 4-coil, 16-spoke frame (7 Newton x 30 CG)"}


def cpu_seconds() -> float:
    """User + system CPU time of this process (all threads), to report the threads the oracle really used."""
    import resource
    ru = resource.getrusage(resource.RUSAGE_SELF)
    return ru.ru_utime + ru.ru_stime


def run_reference(args, rank, world):
    if rank != 0:
        return None
    import numpy as np
    W = synth_workload()
    O, s, fr, y, x0 = _oracle_problem(W)
    c = O.coils(s, x0)
    r0, _ = O.residual(s, fr.mask, y, x0)
    b = O.adjoint(s, fr.mask, x0, r0, c)
    alpha = W.alpha0
    r = b.copy()
    p = r.copy()
    dx = np.zeros_like(b)
    rr = O.inner(r, r).real

    # the CG iterations one oracle frame executes (solves stop at the rounding floor): one frame reconstructed
    # once, untimed, to count them
    stops = []
    O.irgnm(s, fr.mask, y, x0, None, W.newton_steps, W.cg_iters, cg_stops=stops)
    iters = sum(W.cg_iters if st < 0 else st + 1 for st in stops)

    def one_iter():
        nonlocal r, p, dx, rr
        q = O.normal(s, fr.mask, x0, p, alpha, c)
        pq = O.inner(p, q).real
        a = rr / pq if pq > 0 else 0.0
        dx = dx + a * p
        r = r - a * q
        rn = O.inner(r, r).real
        p = r + (rn / rr if rr else 0.0) * p
        rr = rn

    for _ in range(args.warmup):
        one_iter()
    c0 = cpu_seconds()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one_iter()
    wall = time.perf_counter() - t0
    cores = max(1, round((cpu_seconds() - c0) / wall))
    dt = wall / args.steps
    per_frame = dt * (iters + W.newton_steps)   # + about one iteration's work per Newton step (residual, rhs)
    value = 1.0 / per_frame
    return {
        "metric": METRIC, "value": round(value, 6), "unit": "frames/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c128", "data": "synthetic", "impl": "reference",
        "config": {"workload": "real-time radial series: 384x384 grid, 10 coils, 13 spokes, 7 Newton x 30 CG",
                   "sample": "one CG iteration of Newton step 0 per step"},
        "cpu_baseline": {"value": round(value, 6), "unit": "frames/s", "cores": cores, "kind": "oracle",
                         "sample": f"each step = one CG iteration (normal operator + updates) at 384x384, 10 coils; "
                                   f"frame = {iters} + {W.newton_steps} such iterations (the CG iterations one oracle "
                                   f"frame executes, solves stopping at the rounding floor, plus one per Newton step "
                                   f"for the residual and right-hand side)"},
        "e2e": {"value": round(value, 6), "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def synth_workload():
    from paper_1301_1215_gb300 import synth
    return synth.WORKLOADS[WORKLOAD]


CG_KERNEL_ORDER = ("row p-update/W^-1", "col W^-1/C/FFT", "row PSF", "col FFT^-1/C^H/FFT", "row W^-H+alpha p",
                   "cg step")


def write_traffic(rep: str) -> None:
    """profiles/traffic.json from an ncu report holding, in launch order, the CG kernels of one
    nlinv_profile_cg iteration (dram__bytes_read.sum + dram__bytes_write.sum per launch)."""
    import csv
    import io
    out = subprocess.run(["ncu", "-i", rep, "--page", "raw", "--csv"], capture_output=True, text=True, check=True).stdout
    rows = list(csv.reader(io.StringIO(out)))
    hdr, units, data = rows[0], rows[1], rows[2:]
    scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}
    ri, wi = hdr.index("dram__bytes_read.sum"), hdr.index("dram__bytes_write.sum")
    kernels = {}
    for name, d in zip(CG_KERNEL_ORDER, data):
        kernels[name] = int(float(d[ri]) * scale[units[ri]] + float(d[wi]) * scale[units[wi]])
    doc = {"csrc_digest": csrc_digest(), "source": os.path.basename(rep), "kernels": kernels,
           "note": "ncu flushes caches per replay pass: DRAM bytes of one cold launch"}
    with open(os.path.join(ROOT, "profiles", "traffic.json"), "w") as f:
        json.dump(doc, f, indent=1)
    print(json.dumps(doc))


def batch_shapes(nframes: int = 64, seed: int = 1004):
    """Seeded uneven workload: grid side from {128, 192, 256, 320, 384}, coils 4..16, spokes 9..31 per frame."""
    from paper_1301_1215_gb300 import synth
    return synth.uneven_batch_shapes(nframes, seed)


def frame_bytes(n: int, J: int, newton: int, cg: int) -> float:
    """Algorithmic bytes of one reconstruction: the CG kernels' compulsory bytes per iteration (cg_bytes) times the
    iterations, plus about one iteration's worth per Newton step for the residual and right-hand side."""
    per_iter = sum(cg_bytes(n, J, n // 4).values())
    return per_iter * newton * (cg + 1)


def batch_inputs(torch, dev, shapes, snr_db=30.0):
    """Noisy data of the uneven batch: per frame a seeded phantom and coils, its own radial mask, y = P FFT(M rho
    c_j) from the library's simulation kernel plus complex Gaussian noise at snr_db on the sampled points."""
    import numpy as np
    from paper_1301_1215_gb300 import synth
    from paper_1301_1215_gb300.nlinv import Nlinv
    gen = torch.Generator(device=dev)
    gen.manual_seed(1004)
    ys, ms = [], []
    for i, (n, J, S) in enumerate(shapes):
        fr = synth.make_frame(n, J, S, seed=5000 + i)
        m = torch.from_numpy(fr.mask).to(dev)
        with Nlinv(n, J, device=dev) as ctx:
            y = ctx.simulate(torch.from_numpy(fr.rho.astype(np.complex64)).to(dev),
                             torch.from_numpy(fr.coils.astype(np.complex64)).to(dev), m)
        power = float((y.abs() ** 2).sum().item()) / (float(m.sum().item()) * J)
        sigma = synth.noise_sigma(power, snr_db)
        noise = torch.randn((J, n, n, 2), generator=gen, device=dev) * (sigma * 0.5 ** 0.5)
        y += torch.view_as_complex(noise) * m
        ys.append(y)
        ms.append(m)
    torch.cuda.synchronize()
    return ys, ms


def batch_compare(torch, dev, K=3, Wm=1, profile_only=False):
    """The uneven batch workload (64 frames, grid side 128..384, 4..16 coils, 9..31 spokes, 7 Newton x 30 CG):
    the batched, graph-captured form (one launch per pass and grid side) against the plain per-frame form (one
    context and graph per frame, frames one after another), both timed with CUDA events over K whole batches after
    Wm untimed ones (the ~0.4 GB working set is larger than L2), plus a parity spot check: one frame per grid side,
    batched result against the plain one."""
    from paper_1301_1215_gb300.nlinv import Nlinv, NlinvBatch
    W = synth_workload()
    shapes = batch_shapes()
    ys, ms = batch_inputs(torch, dev, shapes)
    opts = dict(newton_steps=W.newton_steps, cg_iters=W.cg_iters)
    batch = NlinvBatch([(n, J) for n, J, _ in shapes], device=dev, **opts)
    if profile_only:                       # one untimed reconstruction for a profiler
        batch.reconstruct(ys, ms)
        torch.cuda.synchronize()
        batch.close()
        return None
    for _ in range(Wm):
        batch.reconstruct(ys, ms)
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    batch.stream.wait_stream(torch.cuda.current_stream(dev))
    s.record(batch.stream)
    for _ in range(K):
        xb = batch.reconstruct(ys, ms)
    e.record(batch.stream)
    torch.cuda.synchronize()
    t_batch = s.elapsed_time(e) / K / 1e3
    launches = batch.launch_count
    # each batched CG kernel alone (all sides, back to back): its algorithmic bytes over all frames / duration, in
    # the HBM-bound regime (the frames' ~3.7 GB of workspaces are far larger than L2)
    bprof = batch.profile_cg(reps=10)
    batch.close()
    hbm_, _ = peaks()
    bkern = {}
    for kname, kms in bprof.items():
        kb = sum(cg_bytes(n, J, n // 4)[kname] for n, J, _ in shapes)
        bkern[kname] = {"ms": round(kms, 4), "algo_bytes": int(kb), "gbs": round(kb / (kms * 1e-3) / 1e9, 1),
                        "frac": round(kb / (kms * 1e-3) / 1e9 / hbm_, 4)}
    ctxs = [Nlinv(n, J, device=dev, **opts) for n, J, _ in shapes]
    xp = [None] * len(ctxs)
    for i, (c, y, m) in enumerate(zip(ctxs, ys, ms)):
        for _ in range(Wm):
            xp[i] = c.reconstruct(y, m)
    torch.cuda.synchronize()
    s.record()
    for _ in range(K):
        for i, (c, y, m) in enumerate(zip(ctxs, ys, ms)):
            xp[i] = c.reconstruct(y, m)
    e.record()
    torch.cuda.synchronize()
    t_plain = s.elapsed_time(e) / K / 1e3
    for c in ctxs:
        c.close()
    spot, finite = {}, True
    for i, (n, J, _) in enumerate(shapes):
        finite = finite and bool(torch.isfinite(torch.view_as_real(xb[i])).all().item())
        if n not in spot:
            d = (xb[i] - xp[i]).abs().pow(2).sum().sqrt() / xp[i].abs().pow(2).sum().sqrt()
            spot[n] = {"frame": i, "coils": J, "rel_l2_batched_vs_plain": float(f"{float(d.item()):.3e}")}
    # the autotuner on one frame of every grid side (single-frame contexts): does any side want other tile shapes
    # than the compiled ones the batched kernels use?
    tuning = {}
    for i, (n, J, _) in enumerate(shapes):
        if n in tuning:
            continue
        with Nlinv(n, J, device=dev, **opts) as c:
            t = c.autotune(ys[i], ms[i], reps=3)
        default = next(cd for cd in t["candidates"] if cd["stage"] == 0)     # stage 0 starts from the defaults
        tuning[n] = {"coils": J, "chosen": {k: t[k] for k in ("split_n1", "col_strip", "row_blocks_per_sm",
                                                               "vec_blocks_per_sm", "pdl", "ms_per_frame")},
                     "compiled_default_ms": default["ms_per_frame"],
                     "candidates": [[cd["stage"], cd["split_n1"], cd["col_strip"], cd["row_blocks_per_sm"],
                                     cd["vec_blocks_per_sm"], int(cd["pdl"]), cd["ms_per_frame"]]
                                    for cd in t["candidates"]]}
    nf = len(shapes)
    total_bytes = sum(frame_bytes(n, J, W.newton_steps, W.cg_iters) for n, J, _ in shapes)
    comp_bytes = sum(compulsory_bytes(n, J) * W.newton_steps * W.cg_iters for n, J, _ in shapes)
    hbm, src = peaks()
    return {
        "workload": "64 independent frames, seeded: grid side {128..384}, 4-16 coils, 9-31 spokes, 30 dB noise, "
                    "7 Newton x 30 CG",
        "batched": {"value": round(nf / t_batch, 3), "unit": "frames/s", "ms_per_batch": round(t_batch * 1e3, 3),
                    "form": "one launch per pass and grid side, sides as parallel branches of one CUDA graph"},
        "plain_per_frame": {"value": round(nf / t_plain, 3), "unit": "frames/s", "ms_per_batch": round(t_plain * 1e3, 3),
                            "form": "one context and graph per frame, frames in sequence"},
        "batched_over_plain": round(t_plain / t_batch, 3),
        "steps": K, "warmup": Wm, "gpu_launches_per_batch": int(launches),
        "algo_gbs": round(total_bytes / t_batch / 1e9, 1), "algo_frac": round(total_bytes / t_batch / 1e9 / hbm, 4),
        "compulsory_gbs": round(comp_bytes / t_batch / 1e9, 1),
        "compulsory_frac": round(comp_bytes / t_batch / 1e9 / hbm, 4), "peak": hbm, "peak_source": src,
        "parity_spot_check": spot, "finite": finite,
        "l2": "inputs larger than L2 (the 64 frames' workspaces hold ~3.7 GB)",
        "kernels_hbm_bound": {"note": "each batched kernel of one CG iteration launched alone for all sides, 10 times "
                                      "back to back (nlinv_batch_profile_cg); algorithmic bytes as in "
                                      "roofline.kernels, summed over the 64 frames; frac of the measured HBM peak",
                              "kernels": bkern},
        "autotune_per_side": {"note": "nlinv_autotune on one frame of each side (single-frame context); candidates: "
                                      "[stage, split_n1, col_strip, row_blocks_per_sm, vec_blocks_per_sm, pdl, "
                                      "ms_per_frame]; the batched kernels run the compiled split and strip",
                              "sides": tuning},
    }


GOLDEN_512 = os.path.join(ROOT, "tests", "golden", "precision_512.npz")


def precision_compare(torch, dev, K=3, Wm=1):
    """The precision workload (512 x 512 grid, 16 coils, 32 spokes, 8 Newton x 30 CG) with FP32 radix-16 stages and
    with the split-BF16 tensor-core stages: ms per frame (CUDA events over K frames after Wm, each from the same
    start value; the ~0.3 GB working set is larger than L2) and the relative L2 error of every Newton iterate (on
    the stored structured sample) and of the final image against the complex128 oracle's run stored in
    tests/golden/precision_512.npz.  The data are simulated here with the library's own kernel plus the stored
    run's seeded noise (they differ from the oracle's data by FP32 rounding)."""
    import numpy as np
    from paper_1301_1215_gb300 import synth
    from paper_1301_1215_gb300.nlinv import Nlinv
    if not os.path.exists(GOLDEN_512):
        return {"unavailable": "tests/golden/precision_512.npz is missing"}
    g = np.load(GOLDEN_512)
    n, J, spokes, seed, newton, cg = (int(v) for v in g["meta"])
    fr = synth.make_frame(n, J, spokes, seed=seed)
    tm = torch.from_numpy(fr.mask).to(dev)
    with Nlinv(n, J, device=dev) as c0:
        y = c0.simulate(torch.from_numpy(fr.rho.astype(np.complex64)).to(dev),
                        torch.from_numpy(fr.coils.astype(np.complex64)).to(dev), tm)
    power = float((y.abs() ** 2).sum().item()) / (float(tm.sum().item()) * J)
    y += torch.from_numpy((synth.noise_sigma(power, 30.0) * fr.noise).astype(np.complex64)).to(dev) * tm
    idx = g["sample_index"]
    h = n // 2
    out = {"workload": f"{n}x{n} grid, {J} coils, {spokes} spokes, {newton} Newton x {cg} CG, 30 dB noise",
           "reference": "complex128 oracle, stored by tests/golden/make_precision_512.py",
           "error_metric": "relative L2: per Newton iterate on the stored sample (rho on Omega every 4th pixel, "
                           "central 8x8 k-space block of every chat_j); final rho on Omega; final display image"}
    for name, tc in (("fp32", False), ("tensor_core_split_bf16", True)):
        with Nlinv(n, J, newton_steps=newton, cg_iters=cg, tensor_dft=tc, device=dev) as ctx:
            for _ in range(Wm):
                ctx.reconstruct(y, tm)
            torch.cuda.synchronize()
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ctx.stream.wait_stream(torch.cuda.current_stream(dev))
            s.record(ctx.stream)
            for _ in range(K):
                ctx.reconstruct(y, tm)
            e.record(ctx.stream)
            torch.cuda.synchronize()
            ms = s.elapsed_time(e) / K
            xN, ck = ctx.reconstruct_checkpoints(y, tm)
            img = ctx.image(xN).cpu().numpy()
            ck = ck.cpu().numpy()

        def rel(a, b):
            return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))
        rho = np.fft.fftshift(ck[-1][0])[h - n // 4: h + n // 4, h - n // 4: h + n // 4]
        out[name] = {"ms_per_frame": round(ms, 3), "frames_per_s": round(1e3 / ms, 2),
                     "per_newton_rel_l2": [float(f"{rel(ck[k].ravel()[idx], g['samples'][k]):.3e}")
                                           for k in range(1, newton + 1)],
                     "final_rho_rel_l2": float(f"{rel(rho, g['rho_omega']):.3e}"),
                     "final_image_rel_l2": float(f"{rel(img, g['image']):.3e}")}
    out["tensor_core_over_fp32_speed"] = round(out["fp32"]["ms_per_frame"] /
                                               out["tensor_core_split_bf16"]["ms_per_frame"], 3)
    return out


def run_batch(args):
    import torch
    from paper_1301_1215_gb300.build import build

    build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    K, Wm = max(1, min(args.steps, 5)), max(1, min(args.warmup, 2))
    if args.batch_profile:
        batch_compare(torch, dev, profile_only=True)
        return {"impl": "ours", "profile_run": "one batched reconstruction of the 64 frames, untimed"}
    b = batch_compare(torch, dev, K=K, Wm=Wm)
    return {
        "metric": "NLINV batched frames/s, 64 uneven frames (grid 128-384, 4-16 coils)", "value": b["batched"]["value"],
        "unit": "frames/s", "n_gpus": 1, "steps": K, "warmup": Wm, "ms_per_step": b["batched"]["ms_per_batch"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64 (f32 complex; f64 CG scalars)",
        "data": "synthetic", "config": {"workload": b["workload"]}, "batch64": b,
        "gpu_launches": int(b["gpu_launches_per_batch"] * K),
    }


def main():
    args = parse()
    if args.write_traffic:
        write_traffic(args.write_traffic)
        return
    if args.workload == "batch64" and args.impl != "reference":
        rank, world, local = dist_env()
        line = run_batch(args)
        if rank == 0:
            print(json.dumps(line), flush=True)
        return
    rank, world, local = dist_env()
    if world > 1:
        import torch
        import torch.distributed as dist
        if args.impl == "reference":
            if rank != 0:
                return
        else:
            torch.cuda.set_device(local)
            dist.init_process_group("nccl")
    if args.impl == "reference":
        line = run_reference(args, rank, world)
    else:
        line = run_ours(args, rank, world, local)
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)
    if world > 1 and args.impl != "reference":
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
