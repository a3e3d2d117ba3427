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
time of the steps). L2 (126 MB) is flushed between steps by writing a buffer of
twice its size outside the timed region; within a frame the iterations run back to back
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
FUSED_DRAM_BYTES_PER_LAUNCH = 16.32128e6 + 0
# DRAM bytes (read + write) of one whole tracking iteration (its 7 kernels),
# from one ncu capture with the caches carried over between kernels
# (profiles/dram_iteration_track-640x480-300k.md); None once a kernel of the
# iteration changes.
DRAM_BYTES_PER_ITERATION = 0.905728e6 + 5.036544e6
# DRAM bytes of one k_render_fused_pose<16, 3> launch at 1200x680 on the 5M
# Gaussians: 16-bit storage and FP32 storage with the map in Morton order, and
# FP32 storage in the generator's order; ncu, cold cache
# (profiles/dram_fused_precision-1200x680-5M-room.md); None for other builds.
PREC16_FUSED_DRAM_BYTES_PER_LAUNCH = 104.30976e6 + 2.601984e6
PREC32_FUSED_DRAM_BYTES_PER_LAUNCH = 104.235264e6 + 3.001088e6
PREC32_GIVEN_ORDER_FUSED_DRAM_BYTES_PER_LAUNCH = None  # not captured for the current kernel
# DRAM bytes of one step's FULL backward (k_render_bwd<16, FULL> + the
# projection adjoint k_project_bwd) on the mapping window and on the uneven
# batch, per-tile schedule at tile 16, staging batch 512 (the blend backward's
# bytes at 256 measured the same within 0.1%), maps in Morton order; ncu, one
# pass per launch (profiles/dram_bwd_full_mapping-uneven.md); None for other
# configurations and once either kernel changes.
MAP_BWD_DRAM_BYTES_PER_STEP = (280.562944e6 + 36.974080e6) + (140.781056e6 + 27.464192e6)
UNEVEN_BWD_DRAM_BYTES_PER_STEP = (621.399808e6 + 87.581440e6) + (474.705152e6 + 103.974656e6)
FP32_LANES_PER_SM = 128


def _l2_flush_buffer(dev):
    """A device buffer of twice the L2 size (rounded up to a MiB); writing it
    evicts every line of the previous step. Returns (buffer, MiB)."""
    import torch
    l2 = int(getattr(torch.cuda.get_device_properties(dev), "L2_cache_size", 0) or (126 << 20))
    mib = -(-2 * l2 // (1 << 20))
    return torch.empty(mib << 20, dtype=torch.uint8, device=dev), mib


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
    p.add_argument("--batch", type=int, default=0, choices=(0, 256, 512),
                   help="mapping/uneven: list entries staged per CTA batch (0 = 512)")
    p.add_argument("--sched", choices=("auto", "tile", "persistent"), default="auto",
                   help="mapping/uneven: one CTA per tile or persistent CTAs (auto: the autotuner's pick for "
                        "uneven, per tile for mapping)")
    p.add_argument("--no-graph", action="store_true", help="mapping/uneven: launch the step eagerly")
    p.add_argument("--storage", choices=("16bit", "fp32"), default="16bit",
                   help="precision: the Gaussians in 16-bit storage or in plain FP32")
    p.add_argument("--order", choices=("morton", "given"), default=None,
                   help="the map in Morton order (gs_spatial_order, once before timing) or in the "
                        "generator's order (default: given for track, morton otherwise)")
    a = p.parse_args()
    if a.order is None:
        a.order = "given" if a.workload == "track" else "morton"
    return a


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
    if a.order == "morton":
        g = morton_ordered(g, dev)
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
    flush, flush_mib = _l2_flush_buffer(dev)

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
                       f"the tracking of frame k; the {flush_mib} MiB L2 flush between frames is inside the timed region"}

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
        # the library's build: 3 CTAs per SM at tile 16, 1 otherwise
        minb = 3 if a.tile == 16 else 1
        kname, flop, traffic = f"k_render_fused_pose<{a.tile}, {minb}>", FWD_FLOP_PER_CONTRIB + BWD_FLOP_PER_CONTRIB, \
            (FUSED_DRAM_BYTES_PER_LAUNCH if a.tile == 16 else None)
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
    # per-stage device time of an iteration, from one frame after the timed
    # region, captured with an event node around each library call
    f_last = my_frames[a.warmup + a.steps - 1]
    stage_ms = tr.stage_ms(tcol[f_last], tdep[f_last], starts_t[f_last])

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
            "config": {"workload": WORKLOAD, "width": 640, "height": 480, "gaussians": int(g.n), "map_order": a.order,
                       "iters_per_frame": ITERS, "step": "one tracked frame (30 iterations)", "tile": a.tile,
                       "l2": f"flushed between steps ({flush_mib} MiB write, twice the L2, untimed)", "parallelism": f"replicas x{ws}",
                       "ms_per_iteration": total_ms / (a.steps * ITERS), "wall_s": wall,
                       "pairs_per_iteration": int(tr.rast.read_status()[1]),
                       "contributions_per_iteration": E, "bwd_share_of_step": bwd_share,
                       "stage_ms": stage_ms},
            "roofline": roof, "hbm": hbm, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
            "context": "paper: 7.89 ms x 15 tracking iterations on an RTX 4090 (Table 5, Replica office-0)"}
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


# ---------------------------------------------------------------- batches
def _oracle_frame_grad_rate(scene, cam, T, tc, td, loss_w, frames=1):
    """The oracle's FULL gradient (forward + analytic adjoint to every
    parameter and the pose) of one frame, timed on this host's cores."""
    import numpy as np

    import oracle
    L = oracle.LossSpec(loss_w["w_color"], loss_w["w_depth"], loss_w.get("w_unc", 0.0), 0.0, 0.0,
                        np.asarray(tc, np.float64), np.asarray(td, np.float64), w_align=loss_w.get("w_align", 0.0))
    t0 = time.perf_counter()
    for _ in range(frames):
        oracle.grad(scene, cam, T, L)
    return frames / (time.perf_counter() - t0), oracle.threads()


def run_batch(a):
    """Mapping window (8 keyframes) or uneven batch (16 mixed frames): one step =
    project + bin + forward + FULL backward (fused loss) over the whole batch,
    captured once in a CUDA graph and replayed (--no-graph: launched eagerly).
    Mapping under torchrun shards the window by keyframe: every rank steps its
    own frames and one NCCL all-reduce sums the parameter gradients (fixed
    8-frame window: strong scaling)."""
    import numpy as np
    import torch

    import synth
    from paper_2403_16095_b300 import Gaussians, Rasterizer, autotune
    from paper_2403_16095_b300 import _abi as A
    from paper_2403_16095_b300.build import build
    from paper_2403_16095_b300.shard import ShardedWindow, allreduce_gaussian_grads
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
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
    if a.order == "morton":
        g = morton_ordered(g, dev)
    # the mapping weights of Sec. 4 (Replica): omega_1 colour 0.7, omega_3 geo 0.25,
    # omega_4 align 0.25, omega_6 var 0.15 (SSIM and L_iso are off the rasterizer)
    loss_w = dict(w_color=0.7, w_depth=0.25, w_unc=0.15, w_align=0.25)
    loss = dict(loss_w, target_color=tcol, target_depth=tdep)
    sched_of = {"tile": A.GS_SCHED_TILE, "persistent": A.GS_SCHED_PERSISTENT}
    tile, batch, sched, tune = a.tile, a.batch, sched_of.get(a.sched, A.GS_SCHED_TILE), None
    if a.workload == "uneven" and a.sched == "auto":
        (tile, batch, sched), times = autotune(cams, g, Tt, tdep, mode=A.GS_MODE_FULL, loss=loss)
        tune = {f"tile{t}/batch{b}/{'persistent' if s_ else 'per-tile'}": ms for (t, b, s_), ms in times.items()}
    elif a.sched == "auto":
        sched = A.GS_SCHED_TILE
    grads = {k: torch.empty_like(getattr(g, k)) for k in names}
    if a.workload == "mapping":
        sw = ShardedWindow(cams, g.n, Tt, tcol, tdep, rank=rank, world=ws, tile=tile, loss_weights=loss_w,
                           batch=batch, sched=sched)
        sw.prepare(g)
        r, my_cams, my_T, my_loss, my_dep = sw.rast, sw.cams, sw.T_cw, sw.loss, sw.target_depth
    else:
        r = Rasterizer(cams, g.n, tile=tile, mode=A.GS_MODE_FULL, batch=batch, sched=sched)
        r.render(g, Tt, tdep)
        r.set_capacity(int(r.read_status()[1] * 1.25) + 4096)
        my_cams, my_T, my_loss, my_dep = cams, Tt, loss, tdep
    flush, flush_mib = _l2_flush_buffer(dev)
    # separate projection and binning calls: on multi-frame batches the count
    # kernel (8 records per thread) beats counting inside the projection
    stages = ("project", "bin", "forward", "backward")

    def eager_step():
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        ev[0].record()
        r.project(g, my_T)
        ev[1].record()
        r.bin()
        ev[2].record()
        r.forward(my_dep)
        ev[3].record()
        r.backward(obs_depth=my_dep, loss=my_loss, g=g, T_cw=my_T, grads=grads)
        ev[4].record()
        return ev

    for _ in range(a.warmup):
        flush.zero_()
        eager_step()
    torch.cuda.synchronize()
    assert r.read_status()[0] == 0
    # per-stage times and the work counts from eager steps (outside the timed line)
    per = {s_: [] for s_ in stages}
    contrib = []
    for _ in range(min(a.steps, 5)):
        flush.zero_()
        ev = eager_step()
        ev[-1].synchronize()
        for i, s_ in enumerate(stages):
            per[s_].append(ev[i].elapsed_time(ev[i + 1]))
        contrib.append(int(r.img["n_contrib"].sum()))
    eager_ms = statistics.mean(sum(per[s_][k] for s_ in stages) for k in range(len(per["project"])))
    graph = None if a.no_graph else r.capture_step(g, my_T, my_dep, my_loss, grads)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    tot = []
    for _ in range(a.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        if graph is not None:
            graph.replay()
        else:
            eager_step()
        if ws > 1:
            allreduce_gaussian_grads(grads, names)
        e1.record()
        e1.synchronize()
        tot.append(e0.elapsed_time(e1))
    barrier()
    clk = clocks.stop()
    if r.read_status()[0] != 0:
        raise RuntimeError("device status set during the timed region")
    total_ms = sum(tot)
    if ws > 1:
        t = torch.tensor([total_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t)
    value = F * a.steps / (total_ms / 1e3)
    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    peaks = _peaks()
    mhz = peaks.get("sm_max_mhz", 2032.0)
    fp32_peak, _ = _fp32_peak(dev, mhz)
    bwd_ms = statistics.mean(per["backward"])
    E = statistics.mean(contrib)
    achieved = E * BWD_FULL_FLOP_PER_CONTRIB / (bwd_ms * 1e-3) / 1e12
    n_pix = sum(int(c.width) * int(c.height) for c in cams)
    metric = {"mapping": "mapping keyframe-iterations/sec (fwd+FULL bwd), 8x640x480 window, 1M Gaussians",
              "uneven": "frames/sec (fwd+FULL bwd), 16 mixed-resolution frames in one batch, 2M Gaussians"}[a.workload]
    cpu = None
    if not a.no_cpu_baseline:
        # the oracle's FULL gradient of one frame of the batch (the first 640x480 one)
        f0 = next(f for f, c in enumerate(cams) if int(c.width) == 640)
        off = sum(int(c.width) * int(c.height) for c in cams[:f0])
        hw = int(cams[f0].width) * int(cams[f0].height)
        tc0 = tcol[3 * off: 3 * (off + hw)].view(3, int(cams[f0].height), int(cams[f0].width)).cpu().numpy()
        td0 = tdep[off: off + hw].view(int(cams[f0].height), int(cams[f0].width)).cpu().numpy()
        sc_p = synth.Scene(*(pert[k] for k in names))
        rate, cores = _oracle_frame_grad_rate(sc_p, cams[f0], np.asarray(poses[f0], np.float64), tc0, td0, loss_w)
        cpu = {"value": rate, "unit": "frames/s", "cores": cores, "kind": "oracle",
               "sample": f"the FP64 oracle's forward + analytic FULL gradient of frame {f0} (640x480) of the batch, "
                         f"{g.n // 1000}k Gaussians, one frame"}
    sched_name = "persistent" if sched == A.GS_SCHED_PERSISTENT else "per-tile"
    # the captured configurations only (the autotuner's picks on the default workloads)
    cap_bytes = {"mapping": MAP_BWD_DRAM_BYTES_PER_STEP, "uneven": UNEVEN_BWD_DRAM_BYTES_PER_STEP}[a.workload]
    bwd_traffic = (cap_bytes if (sched_name == "per-tile" and tile == 16 and a.order == "morton" and ws == 1)
                   else None)
    bwd_traffic_src = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of k_render_bwd + k_project_bwd, "
                       "one step, caches flushed before each launch" if bwd_traffic else
                       "not captured for this configuration")
    line = {"metric": metric, "value": value, "unit": "frames/s", "n_gpus": ws, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": total_ms / a.steps, "higher_is_better": True,
            "scaling": "strong" if a.workload == "mapping" else "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{a.workload}-{F}frames-{g.n // 1000}k", "frames": F, "pixels": n_pix,
                       "gaussians": int(g.n), "map_order": a.order, "tile": tile, "batch": batch or 512,
                       "sched": sched_name,
                       "launch": "CUDA graph replay" if graph is not None else "eager",
                       "parallelism": f"keyframe shards x{ws}" if a.workload == "mapping" else "single batch",
                       "autotune_ms": tune, "l2": f"flushed between steps ({flush_mib} MiB write, twice the L2, untimed)",
                       "stage_ms_eager": {s_: statistics.mean(v) for s_, v in per.items()},
                       "eager_ms_per_step": eager_ms,
                       "pairs": int(r.read_status()[1]), "contributions": E},
            "roofline": {"kernel": f"k_render_bwd<{tile},FULL> + k_project_bwd", "bound": "alu",
                         "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                         "traffic": bwd_traffic, "traffic_source": bwd_traffic_src,
                         "flop_per_contribution": BWD_FULL_FLOP_PER_CONTRIB, "avg_launch_ms": bwd_ms},
            # projection, 5 binning kernels, forward, FULL backward, projection adjoint
            "cpu_baseline": cpu, "gpu_launches": 9 * a.steps, "clocks": clk}
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def morton_ordered(g, dev):
    """A copy of the FP32 map g with its Gaussians in Morton order of their
    means (gs_spatial_order), gathered once before any timed region."""
    import torch
    from paper_2403_16095_b300 import Gaussians
    from paper_2403_16095_b300 import _abi as A
    perm = torch.empty(g.n, dtype=torch.int32, device=dev)
    ws_sort = torch.empty(max(1, A.gs_spatial_order_workspace_size(g.n)), dtype=torch.uint8, device=dev)
    st = torch.zeros(4, dtype=torch.int32, device=dev)
    A.gs_spatial_order(g.means, perm, ws_sort, st)
    if int(st[0]) != 0:
        raise RuntimeError("gs_spatial_order set the device status")
    idx = perm.long()
    names = ("means", "log_scales", "quats", "opacity_logit", "colors", "nu")
    return Gaussians(*(getattr(g, k)[idx].contiguous() for k in names))


def run_precision(a):
    """Tracking at 1200x680 on 5M Gaussians, 30 iterations per frame in a CUDA
    graph, over the workload's 100 seeded frames (--steps 100 covers them all),
    with the Gaussians in 16-bit storage (BF16 attributes, per-chunk fixed-point
    means; --storage 16bit) or in plain FP32 (--storage fp32), so that the two
    forms are measured on the same GPU at the same shape."""
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
    packed = a.storage == "16bit"
    morton = a.order == "morton"
    if packed:
        gt = pack_bf16(g32, spatial=morton)
    elif morton:  # the same record order as the 16-bit form
        gt = morton_ordered(g32, dev)
    else:
        gt = g32
    frames = list(range(a.warmup + a.steps))
    n_pose = len(poses)
    # targets: the FP32 field rendered at the true poses (device-resident inputs)
    r0 = Rasterizer([cam], g32.n, tile=a.tile, mode=A.GS_MODE_FWD)
    tcol, tdep = {}, {}
    for f in sorted(set(f % n_pose for f in frames)):
        r0.render(g32, torch.from_numpy(np.asarray(poses[f], np.float32)).to(dev).reshape(-1))
        tcol[f], tdep[f] = r0.img["color"].clone(), r0.img["depth"].clone()
    del r0
    starts = {f: torch.from_numpy(synth.jitter_pose(poses[f], seed=1005 * 100 + f)).to(dev)
              for f in sorted(set(f % n_pose for f in frames))}
    tr = Tracker(gt, cam, tile=a.tile, iters=ITERS, graph=True, timing=True, timing_every=TIMING_EVERY)
    tr.prepare(tcol[0], tdep[0], starts[0], headroom=1.6)
    flush, flush_mib = _l2_flush_buffer(dev)
    for f in frames[:a.warmup]:
        flush.zero_()
        tr.set_frame(tcol[f % n_pose], tdep[f % n_pose], starts[f % n_pose])
        tr.run()
    torch.cuda.synchronize()
    r_cnt = Rasterizer([cam], g32.n, tile=a.tile, mode=A.GS_MODE_FWD)
    clocks = ClockSampler(local)
    clocks.start()
    tot, bwd, contrib = [], [], []
    for k, f in enumerate(frames[a.warmup:]):
        flush.zero_()
        fp = f % n_pose
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        tr.set_frame(tcol[fp], tdep[fp], starts[fp])
        tr.run()
        e1.record()
        e1.synchronize()
        tot.append(e0.elapsed_time(e1))
        bwd.extend(tr.backward_ms())
        if tr.rast.read_status()[0] != 0:
            raise RuntimeError("device status set during the timed region")
        if k % 10 == 0:  # blended entries at the final pose, outside the timed region
            r_cnt.render(gt, tr.T_cw)
            contrib.append(int(r_cnt.img["n_contrib"].sum()))
    clk = clocks.stop()
    total_ms = sum(tot)
    peaks = _peaks()
    mhz = peaks.get("sm_max_mhz", 2032.0)
    fp32_peak, n_sm = _fp32_peak(dev, mhz)
    E = statistics.mean(contrib)
    flop = FWD_FLOP_PER_CONTRIB + BWD_FLOP_PER_CONTRIB
    launch_ms = statistics.mean(bwd)
    achieved = E * flop / (launch_ms * 1e-3) / 1e12
    traffic = ({("16bit", "morton"): PREC16_FUSED_DRAM_BYTES_PER_LAUNCH,
                ("fp32", "morton"): PREC32_FUSED_DRAM_BYTES_PER_LAUNCH,
                ("fp32", "given"): PREC32_GIVEN_ORDER_FUSED_DRAM_BYTES_PER_LAUNCH}.get((a.storage, a.order))
               if a.tile == 16 else None)
    roof = {"kernel": f"k_render_fused_pose<{a.tile}, {3 if a.tile == 16 else 1}>", "bound": "alu", "achieved": achieved,
            "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak, "traffic": traffic,
            "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum, one launch, cold cache",
            "peak_source": f"{n_sm} SMs (device query) x 128 FP32 lanes x 2 x {mhz:.0f} MHz (max SM clock)",
            "flop_per_contribution": flop, "contributions_per_launch": E, "avg_launch_ms": launch_ms,
            "launches": len(bwd)}
    cpu = None
    if not a.no_cpu_baseline:
        import oracle
        field = (oracle.unpack_bf16(gt.anchors.cpu().numpy(), gt.packed.cpu().numpy().view(np.uint16)) if packed
                 else synth.Scene(*(np.asarray(getattr(sc, k), np.float32) for k in names)))
        tc0 = tcol[0].view(3, cam.height, cam.width).cpu().numpy()
        td0 = tdep[0].view(cam.height, cam.width).cpu().numpy()
        n_it = a.cpu_iters or 1
        secs, cores = cpu_oracle_iterations(field, cam, poses, [synth.jitter_pose(poses[0], seed=1005 * 100)], n_it,
                                            (tc0, td0))
        cpu = {"value": n_it / secs, "unit": "iters/s", "cores": cores, "kind": "oracle",
               "sample": f"{n_it} FP64 oracle tracking iteration(s) (forward + analytic pose gradient + Adam) on "
                         f"frame 0, 1200x680, 5M Gaussians ({'decoded 16-bit' if packed else 'FP32'} field)"}
    form = "16-bit storage" if packed else "FP32 storage"
    line = {"metric": f"tracking iters/sec (fwd+pose-bwd) at 1200x680/5M Gaussians, {form}",
            "value": ITERS * a.steps / (total_ms / 1e3), "unit": "iters/s", "n_gpus": 1, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": total_ms / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16 storage, f32 compute" if packed else "f32", "data": "synthetic",
            "config": {"workload": f"precision-1200x680-5M-room-{a.storage}", "gaussians": int(g32.n),
                       "tile": a.tile, "iters_per_frame": ITERS, "frames": len(set(f % n_pose for f in frames[a.warmup:])),
                       "map_order": a.order,
                       "l2": f"flushed between steps ({flush_mib} MiB write, twice the L2, untimed)",
                       "ms_per_iteration": total_ms / (a.steps * ITERS),
                       "pairs_per_iteration": int(tr.rast.read_status()[1])},
            "roofline": roof, "cpu_baseline": cpu,
            "gpu_launches": tr.kernel_launches_per_iteration() * ITERS * a.steps, "clocks": clk}
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
