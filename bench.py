#!/usr/bin/env python
"""Tracking benchmark of the B300 Gaussian rasterizer (CG-SLAM, arXiv 2403.16095).

Workload: 640x480 frames (fx = fy = 600, principal point at the centre), 300,000
Gaussians on the surfaces of a seeded 6x5x3 m room with 20 boxes, 10 ground-truth
poses on a smooth path; each frame starts 2 cm / 1 degree off and runs 30
tracking iterations (project -> bin -> forward -> POSE backward with the fused
uncertainty-weighted L1 colour + depth loss, lambda = {0.2, 1.0} -> FP64 pose
reduction -> Adam step on the pose), captured as one CUDA graph per frame.

A step is one tracked frame (30 iterations). The metric is tracking iterations
per second: value = 30 * steps * ranks / (max over ranks of the summed device
time of the steps). L2 (126 MB) is flushed between steps by writing a 512 MB
buffer outside the timed region; within a frame the iterations run back to back
as tracking does.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload track|mapping|uneven|precision]

The default workload is the tracking one above. The others print their own
line (same keys): ``mapping`` = one mapping iteration over a window of 8
640x480 keyframes of a 1M-Gaussian room (forward + FULL backward to every
parameter and the 8 poses, fused colour/depth/alignment/variance loss);
``uneven`` = 16 frames of mixed resolution (6x 320x240, 6x 640x480, 4x
1200x680) over a 2M-Gaussian two-room scene in one batch, tile size chosen by
the autotuner; ``precision`` = tracking at 1200x680 on 5M Gaussians held in
16-bit storage.

With --gpus N > 1 (under torchrun) every rank tracks its own frames
(independent replicas, no data collective); timing uses a barrier and the max
over ranks. ``--impl reference`` times the FP64 CPU oracle on this host's cores
on a bounded sample of the same workload (one iteration per step).
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
sys.path.insert(0, ROOT)

ITERS = 30
TIMING_EVERY = 10  # iterations between CUDA-event samples of the tracking pass's launch
METRIC = "tracking iters/sec (fwd+pose-bwd) at 640x480/300k Gaussians"
WORKLOAD = "track-640x480-300k-room"
# FP32 operations the adjoint performs per blended (pixel, Gaussian) entry in
# POSE mode: recompute q, G, alpha (13), transmittance recovery (4), channel dot
# product for colour + depth (7), dL/dalpha and the running suffix sum (5),
# gradients of mean2d, conic and depth (21), 6x6 pose-Jacobian contraction (72).
BWD_FLOP_PER_CONTRIB = 122
# FULL mode per blended entry: recompute (13), transmittance recovery (4),
# channel dot product (9 with opacity, U and the median), dL/dalpha and suffix
# sum (5), gradients of mean2d, conic, opacity, depth and colour (21).
BWD_FULL_FLOP_PER_CONTRIB = 52
# DRAM bytes (read + write) of one k_render_bwd<16,POSE> launch: None, since
# the kernel changed after its last ncu capture.
BWD_DRAM_BYTES_PER_LAUNCH = None
# forward per blended entry: offsets (2), q (7), exponent argument (1), opacity x G
# (1), clamp (1), 1 - alpha and T' (2), w (1), colour, depth and nu
# accumulation (10), ex2 (1)
FWD_FLOP_PER_CONTRIB = 26
# DRAM bytes (read + write) of one k_render_fused_pose<16, 3> launch of this
# workload, from one ncu capture of the current kernel
# (profiles/k_render_fused_pose_track-640x480-300k.md, cold cache); None once
# the kernel changes.
FUSED_DRAM_BYTES_PER_LAUNCH = 16.350208e6 + 0
# DRAM bytes (read + write) of one whole tracking iteration (the 6 kernels),
# from one ncu capture with the caches carried over between kernels; None
# until captured for the current build.
DRAM_BYTES_PER_ITERATION = None
FP32_LANES_PER_SM = 128


def _fp32_peak(dev, mhz):
    """FP32 FMA peak in TFLOP/s: SMs (read from the device) x 128 lanes x 2 x clock."""
    import torch
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    return n_sm * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12, n_sm


# Algorithmic HBM bytes of one tracking iteration, per unit (each datum moved
# once, in this library's layouts): every Gaussian's FP32 parameters read
# (60 B); per visible record its 64 B record and 144 B pose Jacobian written,
# its rect + depth read by the binning (20 B) and record + Jacobian read once
# by the tracking pass (208 B); per culled record its 16 B rect written; per
# (Gaussian, tile) pair 12 B written by the fill, read and written once by the
# sort (24 B), and its 4 B index read by the tracking pass; per pixel the RGB-D
# target read (16 B).
HBM_B_PER_GAUSSIAN = 60
HBM_B_PER_VISIBLE = 64 + 144 + 20 + 208
HBM_B_PER_CULLED = 16
HBM_B_PER_PAIR = 12 + 24 + 4
HBM_B_PER_PIXEL = 16


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=("ours", "reference"), default="ours")
    p.add_argument("--tile", type=int, default=16)
    p.add_argument("--workload", choices=("track", "mapping", "uneven", "precision"), default="track")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--unfused", action="store_true", help="forward and backward as two launches per iteration")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-iters", type=int, default=0, help="oracle iterations for the CPU baseline (0 = auto)")
    return p.parse_args()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        # raw samples in a temporary file; the JSON line carries their summary
        self.path = os.path.join(tempfile.gettempdir(), f"gs_bench_clocks_{os.getpid()}_{gpu_index}.csv")

    def start(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        self.f.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": ["no samples"]}
        busy = sorted(sm)[len(sm) // 2:] if len(sm) > 4 else sm  # under load: upper half
        return {"sm_mhz": statistics.median(busy), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- workload
def _workload():
    import synth
    w = synth.workload("track")
    starts = [synth.jitter_pose(T, seed=1002 * 100 + k, trans=0.02, rot_deg=1.0) for k, T in enumerate(w["poses"])]
    return w["scene"], w["cams"][0], w["poses"], starts


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ---------------------------------------------------------------- CPU oracle
def cpu_oracle_iterations(sc, cam, gt_poses, starts, n_iter: int, targets=None):
    """Times ``n_iter`` tracking iterations of the FP64 oracle (forward + analytic
    pose gradient + Adam step) on this host's cores; returns (seconds, cores)."""
    import numpy as np

    import oracle
    cores = oracle.threads()
    if targets is None:
        ref = oracle.render(sc, cam, gt_poses[0])
        targets = (ref["color"], ref["depth"])
    L = oracle.LossSpec(0.2, 1.0, 0.0, 0.0, 0.025, targets[0], targets[1])
    st = np.zeros(25)
    T = np.asarray(starts[0], np.float64)
    st[:9] = T[:, :3].reshape(-1)
    st[9:12] = T[:, 3]
    t0 = time.perf_counter()
    for _ in range(n_iter):
        Tc = np.c_[st[:9].reshape(3, 3), st[9:12]]
        g = oracle.grad(sc, cam, Tc, L)
        oracle.adam_step(st, g["pose"])
    return time.perf_counter() - t0, cores


def cpu_baseline(sc, cam, gt, starts, n_all: int, n_one: int):
    """The oracle's tracking iteration timed on all host cores (n_all
    iterations) and on one core (n_one), plus the brute-force O(HW N) render of
    the 128x96 / 2k scene; the oracle as it stands, on a bounded sample."""
    import oracle
    import synth
    ref = oracle.render(sc, cam, gt[0])
    tg = (ref["color"], ref["depth"])
    cpu_oracle_iterations(sc, cam, gt, starts, 1, tg)  # warm (page-in, thread pool)
    secs, cores = cpu_oracle_iterations(sc, cam, gt, starts, n_all, tg)
    out = {"value": n_all / secs, "unit": "iters/s", "cores": cores, "kind": "oracle",
           "sample": f"{n_all} FP64 oracle tracking iterations (forward + analytic pose gradient + Adam) on "
                     f"frame 0, 640x480, 300k Gaussians, rect-scatter lists"}
    if n_one > 0:
        prev = oracle.threads()
        oracle.set_threads(1)
        try:
            s1, _ = cpu_oracle_iterations(sc, cam, gt, starts, n_one, tg)
        finally:
            oracle.set_threads(prev)
        out["single_core"] = {"value": n_one / s1, "unit": "iters/s", "cores": 1,
                              "sample": f"{n_one} of the same iterations on one core"}
    tsc, tcam, tT = synth.tiny_scene()
    t0 = time.perf_counter()
    oracle.render(tsc, tcam, tT, mode="brute")
    out["brute_force_tiny"] = {"value": 1.0 / (time.perf_counter() - t0), "unit": "renders/s", "cores": cores,
                               "sample": "one brute-force (every Gaussian per pixel) oracle render, 128x96, 2k"}
    return out


def run_reference(a):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    sc, cam, gt, starts = _workload()
    import oracle
    ref = oracle.render(sc, cam, gt[0])
    targets = (ref["color"], ref["depth"])
    cpu_oracle_iterations(sc, cam, gt, starts, max(0, a.warmup), targets)
    secs, cores = cpu_oracle_iterations(sc, cam, gt, starts, a.steps, targets)
    value = a.steps / secs
    sample = f"{a.steps} oracle tracking iterations (1 per step) on frame 0 of the workload"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": 0,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * secs / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "frames": 1, "iters_per_frame": ITERS},
            "cpu_baseline": {"value": value, "unit": "iters/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU
def run_ours(a):
    import numpy as np
    import torch

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    from paper_2403_16095_b300.build import build
    build()
    from paper_2403_16095_b300 import Gaussians, Rasterizer, Tracker
    from paper_2403_16095_b300 import _abi as A

    sc, cam, gt, starts = _workload()
    n_frames = len(gt)
    g = Gaussians(*(torch.from_numpy(np.ascontiguousarray(getattr(sc, k))).to(dev)
                    for k in ("means", "log_scales", "quats", "opacity_logit", "colors", "nu")))
    my_frames = [(rank + k * ws) % n_frames for k in range(a.warmup + a.steps)]
    # targets: renders at the ground-truth poses of the frames this rank uses
    # (device-resident inputs of the timed region)
    r0 = Rasterizer([cam], g.n, tile=a.tile, mode=A.GS_MODE_FWD)
    tcol, tdep = [None] * n_frames, [None] * n_frames
    for f in sorted(set(my_frames)):
        r0.render(g, torch.from_numpy(np.asarray(gt[f], np.float32)).to(dev).reshape(-1))
        im = r0.frame_images(0)
        tcol[f] = im["color"].clone()
        tdep[f] = im["depth"].clone()
    del r0
    starts_t = [torch.from_numpy(np.asarray(T, np.float64)).to(dev) for T in starts]

    # the tracking pass's launch time is sampled with CUDA events on iterations
    # 0, 10 and 20 of every frame (event nodes on every iteration cost ~9 us each)
    tr = Tracker(g, cam, tile=a.tile, iters=ITERS, graph=True, timing=True, fused=not a.unfused,
                 timing_every=TIMING_EVERY)
    f0 = my_frames[0]
    tr.prepare(tcol[f0], tdep[f0], starts_t[f0], headroom=1.6)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def one_step(f, ev0, ev1):
        ev0.record()
        tr.set_frame(tcol[f], tdep[f], starts_t[f])
        tr.run()
        ev1.record()

    for k in range(a.warmup):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        one_step(my_frames[k], e0, e1)
    torch.cuda.synchronize()
    assert tr.rast.read_status()[0] == 0, "warm-up failed (pair capacity?)"

    r_cnt = Rasterizer([cam], g.n, tile=a.tile, mode=A.GS_MODE_FWD)
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    step_ms, bwd_ms, contrib, t_wall0 = [], [], [], time.perf_counter()
    for k in range(a.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        one_step(my_frames[a.warmup + k], e0, e1)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        bwd_ms.extend(tr.backward_ms())
        # blended entries (the roofline's work unit) of a full-channel forward at the
        # frame's final pose, outside the timed region (the tracker renders only
        # the channels its loss reads)
        r_cnt.render(g, tr.T_cw)
        contrib.append(int(r_cnt.img["n_contrib"].sum()))
        code, _ = tr.rast.read_status()
        if code:
            raise RuntimeError(f"device status {code} during the timed region")
    barrier()
    wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    total_ms = sum(step_ms)
    if ws > 1:
        t = torch.tensor([total_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t)
    value = ITERS * a.steps * ws / (total_ms / 1e3)

    # ---- end to end through the public call with pinned host buffers
    e2e = None
    if not a.no_e2e:
        hc = [None if t is None else t.cpu().pin_memory() for t in tcol]
        hd = [None if t is None else t.cpu().pin_memory() for t in tdep]
        hT = [torch.from_numpy(np.asarray(T, np.float64)).pin_memory() for T in starts]
        outs = [torch.empty(3, 4, dtype=torch.float64).pin_memory() for _ in range(max(a.steps, a.warmup))]
        # frames go through the streaming call: submit() uploads frame k + 1 on a
        # copy stream while frame k is tracked; drain() waits once at the end
        for k in range(a.warmup):
            f = my_frames[k]
            flush.zero_()
            tr.submit(hc[f], hd[f], hT[f], outs[k])
        tr.drain()
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(a.steps):
            f = my_frames[a.warmup + k]
            flush.zero_()  # L2 flush between frames, in stream order, inside the timed region
            tr.submit(hc[f], hd[f], hT[f], outs[k])
        tr.drain()
        e2e_s = time.perf_counter() - t0
        if ws > 1:
            t = torch.tensor([e2e_s], device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            e2e_s = float(t)
        h2d = hc[f0].numel() * 4 + hd[f0].numel() * 4 + 12 * 8
        e2e = {"value": ITERS * a.steps * ws / e2e_s, "unit": "iters/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": 12 * 8 + 4 * 4,
               "note": "per step: frame RGB-D + start pose host->device (pinned), 30 iterations, pose + status "
                       "device->host (pinned), through Tracker.submit/drain: the upload of frame k + 1 overlaps "
                       "the tracking of frame k; the 512 MB L2 flush between frames is inside the timed region"}

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return

    # ---- roofline of the dominant kernel: the fused forward + POSE backward
    # launch (or, with --unfused, the POSE backward alone)
    peaks = _peaks()
    mhz = peaks.get("sm_max_mhz", 2032.0)
    fp32_peak, n_sm = _fp32_peak(dev, mhz)  # TFLOP/s
    bwd_avg_ms = statistics.mean(bwd_ms)
    E = statistics.mean(contrib)
    if tr.fused:
        # the library's build choice: 4 CTAs per SM at >= 800 records per tile, else 3 (tile 16)
        dense = g.n >= 800 * tr.rast.n_tiles
        minb = (4 if dense else 3) if a.tile == 16 else 1
        kname, flop, traffic = f"k_render_fused_pose<{a.tile}, {minb}>", FWD_FLOP_PER_CONTRIB + BWD_FLOP_PER_CONTRIB, \
            (FUSED_DRAM_BYTES_PER_LAUNCH if (a.tile == 16 and not dense) else None)
    else:
        kname, flop, traffic = f"k_render_bwd<{a.tile},POSE>", BWD_FLOP_PER_CONTRIB, \
            (BWD_DRAM_BYTES_PER_LAUNCH if a.tile == 16 else None)
    achieved = E * flop / (bwd_avg_ms * 1e-3) / 1e12
    roof = {"kernel": kname, "bound": "alu", "achieved": achieved, "peak": fp32_peak,
            "unit": "TFLOP/s", "frac": achieved / fp32_peak, "traffic": traffic,
            "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum, one launch, cold cache",
            "peak_source": f"{n_sm} SMs (device query) x 128 FP32 lanes x 2 x {mhz:.0f} MHz (max SM clock)",
            "flop_per_contribution": flop, "contributions_per_launch": E,
            "avg_launch_ms": bwd_avg_ms, "launches": len(bwd_ms),
            "launch_timing": f"CUDA events around the launch on iterations 0, {TIMING_EVERY}, ... of every timed frame"}
    bwd_share = bwd_avg_ms * ITERS * len(step_ms) / sum(step_ms)

    # ---- achieved HBM fraction: algorithmic bytes of an iteration over its time
    visible = int((tr.rast.touched > 0).sum())
    pairs = int(tr.rast.read_status()[1])
    hw = int(cam.width) * int(cam.height)
    alg_bytes = (HBM_B_PER_GAUSSIAN * g.n + HBM_B_PER_VISIBLE * visible + HBM_B_PER_CULLED * (g.n - visible)
                 + HBM_B_PER_PAIR * pairs + HBM_B_PER_PIXEL * hw)
    ms_it = total_ms / (a.steps * ITERS)
    hbm_peak = peaks.get("hbm_gbs")
    hbm = {"algorithmic_bytes_per_iteration": alg_bytes, "achieved_gbs": alg_bytes / (ms_it * 1e-3) / 1e9,
           "peak_gbs": hbm_peak, "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if hbm_peak else None,
           "frac": (alg_bytes / (ms_it * 1e-3) / 1e9) / hbm_peak if hbm_peak else None,
           "visible_records": visible, "pairs": pairs, "pixels": hw,
           "dram_bytes_per_iteration_ncu": DRAM_BYTES_PER_ITERATION,
           "dram_frac_ncu": (DRAM_BYTES_PER_ITERATION / (ms_it * 1e-3) / 1e9 / hbm_peak
                             if (DRAM_BYTES_PER_ITERATION and hbm_peak) else None),
           "bytes": "60 B params per Gaussian; per visible record 64 B record + 144 B Jacobian written, "
                    "20 B read by binning, 208 B read by the tracking pass; 16 B rect per culled record; "
                    "40 B per pair (fill, sort, index read); 16 B RGB-D target per pixel"}

    cpu = None
    if not a.no_cpu_baseline:
        cpu = cpu_baseline(sc, cam, gt, starts, a.cpu_iters or 10, 1)

    launches = tr.kernel_launches_per_iteration() * ITERS * a.steps
    line = {"metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": ws, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": total_ms / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "width": 640, "height": 480, "gaussians": int(g.n),
                       "iters_per_frame": ITERS, "step": "one tracked frame (30 iterations)", "tile": a.tile,
                       "l2": "flushed between steps (512 MB write, untimed)", "parallelism": f"replicas x{ws}",
                       "ms_per_iteration": total_ms / (a.steps * ITERS), "wall_s": wall,
                       "pairs_per_iteration": int(tr.rast.read_status()[1]),
                       "contributions_per_iteration": E, "bwd_share_of_step": bwd_share},
            "roofline": roof, "hbm": hbm, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
            "context": "paper: 7.89 ms x 15 tracking iterations on an RTX 4090 (Table 5, Replica office-0)"}
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


# ---------------------------------------------------------------- batches
def run_batch(a):
    """Mapping window (8 keyframes) or uneven batch (16 mixed frames): one step =
    project + bin + forward + FULL backward (fused loss) over the whole batch."""
    import numpy as np
    import torch

    import synth
    from paper_2403_16095_b300 import Gaussians, Rasterizer, autotune_tile
    from paper_2403_16095_b300 import _abi as A
    from paper_2403_16095_b300.build import build
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build()
    w = synth.workload(a.workload)
    sc, cams, poses = w["scene"], w["cams"], w["poses"]
    F = len(cams)
    names = ("means", "log_scales", "quats", "opacity_logit", "colors", "nu")
    g_true = Gaussians(*(torch.from_numpy(np.ascontiguousarray(getattr(sc, k), np.float32)).to(dev) for k in names))
    Tt = torch.from_numpy(np.ascontiguousarray(np.asarray(poses, np.float32))).to(dev).reshape(-1)
    # targets: the true scene at the true poses; the optimised field is perturbed
    r0 = Rasterizer(cams, g_true.n, tile=16, mode=A.GS_MODE_FWD)
    r0.render(g_true, Tt)
    tcol, tdep = r0.img["color"].clone(), r0.img["depth"].clone()
    del r0
    rng = np.random.default_rng(1000 + (3 if a.workload == "mapping" else 4))
    pert = {k: np.asarray(getattr(sc, k), np.float32).copy() for k in names}
    pert["means"] += rng.normal(0, 0.01, pert["means"].shape).astype(np.float32)
    pert["colors"] = np.clip(pert["colors"] + rng.normal(0, 0.05, pert["colors"].shape), 0, 1).astype(np.float32)
    g = Gaussians(*(torch.from_numpy(pert[k]).to(dev) for k in names))
    # the mapping weights of Sec. 4 (Replica): omega_1 colour 0.7, omega_3 geo 0.25,
    # omega_4 align 0.25, omega_6 var 0.15 (SSIM and L_iso are off the rasterizer)
    loss = dict(w_color=0.7, w_depth=0.25, w_unc=0.15, w_align=0.25, target_color=tcol, target_depth=tdep)
    tile, tune = a.tile, None
    if a.workload == "uneven":
        tile, tune = autotune_tile(cams, g, Tt, tdep, mode=A.GS_MODE_FULL, loss=loss)
    r = Rasterizer(cams, g.n, tile=tile, mode=A.GS_MODE_FULL)
    r.render(g, Tt, tdep)
    r.set_capacity(int(r.read_status()[1] * 1.25) + 4096)
    grads = {k: torch.empty_like(getattr(g, k)) for k in names}
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    # separate projection and binning calls: on multi-frame batches the count
    # kernel (8 records per thread) beats counting inside the projection
    stages = ("project", "bin", "forward", "backward")

    def step():
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        ev[0].record()
        r.project(g, Tt)
        ev[1].record()
        r.bin()
        ev[2].record()
        r.forward(tdep)
        ev[3].record()
        r.backward(obs_depth=tdep, loss=loss, g=g, T_cw=Tt, grads=grads)
        ev[4].record()
        return ev

    for _ in range(a.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    assert r.read_status()[0] == 0
    clocks = ClockSampler(local)
    torch.cuda.synchronize()
    clocks.start()
    per = {s_: [] for s_ in stages}
    tot = []
    contrib = []
    for _ in range(a.steps):
        flush.zero_()
        ev = step()
        ev[-1].synchronize()
        for i, s_ in enumerate(stages):
            per[s_].append(ev[i].elapsed_time(ev[i + 1]))
        tot.append(ev[0].elapsed_time(ev[-1]))
        contrib.append(int(r.img["n_contrib"].sum()))
    clk = clocks.stop()
    if r.read_status()[0] != 0:
        raise RuntimeError("device status set during the timed region")
    total_ms = sum(tot)
    value = F * a.steps / (total_ms / 1e3)
    peaks = _peaks()
    mhz = peaks.get("sm_max_mhz", 2032.0)
    fp32_peak, _ = _fp32_peak(dev, mhz)
    bwd_ms = statistics.mean(per["backward"])
    E = statistics.mean(contrib)
    achieved = E * BWD_FULL_FLOP_PER_CONTRIB / (bwd_ms * 1e-3) / 1e12
    n_pix = sum(int(c.width) * int(c.height) for c in cams)
    metric = {"mapping": "mapping keyframe-iterations/sec (fwd+FULL bwd), 8x640x480 window, 1M Gaussians",
              "uneven": "frames/sec (fwd+FULL bwd), 16 mixed-resolution frames in one batch, 2M Gaussians"}[a.workload]
    line = {"metric": metric, "value": value, "unit": "frames/s", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": total_ms / a.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{a.workload}-{F}frames-{g.n // 1000}k", "frames": F, "pixels": n_pix,
                       "gaussians": int(g.n), "tile": tile, "autotune_ms": tune,
                       "l2": "flushed between steps (512 MB write, untimed)",
                       "stage_ms": {s_: statistics.mean(v) for s_, v in per.items()},
                       "pairs": int(r.read_status()[1]), "contributions": E},
            "roofline": {"kernel": f"k_render_bwd<{tile},FULL> + k_project_bwd", "bound": "alu",
                         "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                         "traffic": None, "flop_per_contribution": BWD_FULL_FLOP_PER_CONTRIB,
                         "avg_launch_ms": bwd_ms},
            # projection, 5 binning kernels, forward, FULL backward, projection adjoint
            "cpu_baseline": None, "gpu_launches": 9 * a.steps, "clocks": clk}
    print(json.dumps(line), flush=True)


def run_precision(a):
    """Tracking at 1200x680 on 5M Gaussians in 16-bit storage (BF16 attributes,
    per-chunk fixed-point means), 30 iterations per frame in a CUDA graph."""
    import numpy as np
    import torch

    import synth
    from paper_2403_16095_b300 import Gaussians, Rasterizer, Tracker, pack_bf16
    from paper_2403_16095_b300 import _abi as A
    from paper_2403_16095_b300.build import build
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build()
    w = synth.workload("precision")
    sc, cam, poses = w["scene"], w["cams"][0], w["poses"]
    names = ("means", "log_scales", "quats", "opacity_logit", "colors", "nu")
    g32 = Gaussians(*(torch.from_numpy(np.ascontiguousarray(getattr(sc, k), np.float32)).to(dev) for k in names))
    pk = pack_bf16(g32, spatial=True)
    frames = list(range(a.warmup + a.steps))
    r0 = Rasterizer([cam], g32.n, tile=a.tile, mode=A.GS_MODE_FWD)
    tcol, tdep = {}, {}
    for f in frames:
        r0.render(g32, torch.from_numpy(np.asarray(poses[f % len(poses)], np.float32)).to(dev).reshape(-1))
        tcol[f], tdep[f] = r0.img["color"].clone(), r0.img["depth"].clone()
    del r0, g32
    starts = {f: torch.from_numpy(synth.jitter_pose(poses[f % len(poses)], seed=1005 * 100 + f)).to(dev)
              for f in frames}
    tr = Tracker(pk, cam, tile=a.tile, iters=ITERS, graph=True, timing=True, timing_every=TIMING_EVERY)
    tr.prepare(tcol[0], tdep[0], starts[0], headroom=1.6)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    for f in frames[:a.warmup]:
        flush.zero_()
        tr.set_frame(tcol[f], tdep[f], starts[f])
        tr.run()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    tot, bwd = [], []
    for f in frames[a.warmup:]:
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        tr.set_frame(tcol[f], tdep[f], starts[f])
        tr.run()
        e1.record()
        e1.synchronize()
        tot.append(e0.elapsed_time(e1))
        bwd.extend(tr.backward_ms())
    clk = clocks.stop()
    if tr.rast.read_status()[0] != 0:
        raise RuntimeError("device status set during the timed region")
    total_ms = sum(tot)
    line = {"metric": "tracking iters/sec (fwd+pose-bwd) at 1200x680/5M Gaussians, 16-bit storage",
            "value": ITERS * a.steps / (total_ms / 1e3), "unit": "iters/s", "n_gpus": 1, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": total_ms / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16 storage, f32 compute", "data": "synthetic",
            "config": {"workload": "precision-1200x680-5M-room", "gaussians": int(pk.n), "tile": a.tile,
                       "iters_per_frame": ITERS, "l2": "flushed between steps (512 MB write, untimed)",
                       "bwd_ms_avg": statistics.mean(bwd), "ms_per_iteration": total_ms / (a.steps * ITERS),
                       "pairs_per_iteration": int(tr.rast.read_status()[1])},
            "cpu_baseline": None, "gpu_launches": tr.kernel_launches_per_iteration() * ITERS * a.steps,
            "clocks": clk}
    print(json.dumps(line), flush=True)


def main():
    a = _args()
    if a.impl == "reference":
        run_reference(a)
    elif a.workload in ("mapping", "uneven"):
        run_batch(a)
    elif a.workload == "precision":
        run_precision(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
