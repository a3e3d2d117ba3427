"""PyTorch-side host code for libgs: device buffers, the call sequence of one
iteration, a ``torch.autograd.Function`` (FULL backward) and the tracking loop
(POSE backward + on-device Adam, captured in a CUDA graph).

PyTorch supplies memory and streams only; every step of the rasterizer runs in
the libgs kernels behind the C ABI (see ``_abi``).
"""
from __future__ import annotations

import math
from typing import Optional, Sequence

import torch

from . import _abi as A
from ._abi import Gaussians, PackedGaussians

CHANNELS = ("color", "depth", "alpha", "unc", "nu_map", "median", "T_final", "n_last", "n_contrib", "median_pos")


def _pix(cams) -> int:
    return int(sum(int(c.width) * int(c.height) for c in cams))


def _tiles(cams, tile) -> int:
    return int(sum(((int(c.width) + tile - 1) // tile) * ((int(c.height) + tile - 1) // tile) for c in cams))


class Rasterizer:
    """Buffers and calls for one batch of frames (fixed cameras) and N Gaussians."""

    def __init__(self, cams: Sequence, n_gaussians: int, tile: int = 16, mode: int = A.GS_MODE_POSE,
                 capacity: Optional[int] = None, jclamp: float = 1.3, nu_cull: float = 0.0,
                 keep_keys: bool = False, dominant: bool = False, channels: str = "all", device=None,
                 batch: int = 0, sched: int = A.GS_SCHED_TILE):
        """channels: "all" renders every channel; "track" only what the tracking
        loss and its POSE backward read (colour, depth, nu map, T_final, n_last),
        which selects the lighter forward kernel. batch (256 or 512; 0 = 512)
        and sched (GS_SCHED_TILE or GS_SCHED_PERSISTENT) choose how the forward
        and the FULL backward stage and schedule tiles; they change speed only."""
        self.cams = list(cams)
        self.F = len(self.cams)
        self.N = int(n_gaussians)
        self.M = self.F * self.N
        self.tile = tile
        self.mode = mode
        self.opts = A.gs_opts(tile, mode, jclamp, nu_cull, batch, sched)
        self.device = torch.device(device or "cuda")
        dev = self.device
        # the persistent kernels' work queue: zero-filled once, left at zero by every launch
        self.queue = torch.zeros(2, dtype=torch.int32, device=dev) if sched == A.GS_SCHED_PERSISTENT else None
        self.rec = torch.empty(self.M * A.GS_REC_FLOATS, dtype=torch.float32, device=dev)
        self.touched = torch.empty(self.M, dtype=torch.int32, device=dev)
        self.jac = (torch.empty(self.M * A.GS_JAC_FLOATS, dtype=torch.float32, device=dev)
                    if mode == A.GS_MODE_POSE else None)
        self.status = torch.zeros(4, dtype=torch.int32, device=dev)
        self.n_tiles = _tiles(self.cams, tile)
        self.ranges = torch.empty(2 * self.n_tiles, dtype=torch.int32, device=dev)
        self.order = torch.empty(self.n_tiles, dtype=torch.int32, device=dev)  # heaviest tiles first
        self.pix_total = _pix(self.cams)
        P = self.pix_total
        self.img = {
            "color": torch.empty(3 * P, dtype=torch.float32, device=dev),
            "depth": torch.empty(P, dtype=torch.float32, device=dev),
            "alpha": torch.empty(P, dtype=torch.float32, device=dev),
            "unc": torch.zeros(P, dtype=torch.float32, device=dev),
            "nu_map": torch.empty(P, dtype=torch.float32, device=dev),
            "median": torch.empty(P, dtype=torch.float32, device=dev),
            "T_final": torch.empty(P, dtype=torch.float32, device=dev),
            "n_last": torch.empty(P, dtype=torch.int32, device=dev),
            "n_contrib": torch.empty(P, dtype=torch.int32, device=dev),
            "median_pos": torch.empty(P, dtype=torch.int32, device=dev),
        }
        if channels == "track":
            for k in ("alpha", "unc", "median", "n_contrib", "median_pos"):
                del self.img[k]
        elif channels != "all":
            raise ValueError(f"channels={channels!r}")
        if dominant:  # dominated pixels for the uncertainty of Eq. 13
            self.img["dom_pos"] = torch.empty(P, dtype=torch.int32, device=dev)
            self.img["dom_weight"] = torch.empty(P, dtype=torch.float32, device=dev)
        self.keep_keys = keep_keys
        self.values = self.keys = self.bin_ws = None
        self.set_capacity(capacity if capacity is not None else max(4096, 2 * self.M))
        if mode != A.GS_MODE_FWD:
            self.per_frame = A.gs_pose_partials_per_frame(mode, self.N, self.cams, tile)
            # double-float partials: [F][per_frame][6][2] (hi, lo)
            self.pose_partials = torch.zeros(self.F * self.per_frame * 12, dtype=torch.float32, device=dev)
            self.pose_grad = torch.zeros(self.F, 6, dtype=torch.float64, device=dev)
            # zero-filled once: the arrival counters in it must start at zero
            self.bwd_ws = torch.zeros(A.gs_render_bwd_workspace_size(self.M, mode), dtype=torch.uint8, device=dev)

    # --------------------------------------------------------------- buffers
    def set_capacity(self, capacity: int) -> None:
        self.capacity = int(capacity)
        dev = self.device
        self.values = torch.empty(self.capacity, dtype=torch.int32, device=dev)
        self.keys = torch.empty(self.capacity, dtype=torch.int64, device=dev) if self.keep_keys else None
        self.bin_ws = torch.empty(A.gs_bin_tiles_workspace_size(self.M, self.capacity), dtype=torch.uint8,
                                  device=dev)

    def reset_status(self) -> None:
        self.status.zero_()

    def read_status(self):
        s = self.status.tolist()
        return int(s[0]), int(s[1])

    # --------------------------------------------------------------- stages
    def project(self, g, T_cw: torch.Tensor, stream=None) -> None:
        """g: Gaussians (FP32) or PackedGaussians (BF16 storage; FWD/POSE modes)."""
        if isinstance(g, PackedGaussians):
            A.gs_project_bf16(g, self.cams, T_cw, self.opts, self.rec, self.touched, self.jac, self.status, stream)
        else:
            A.gs_project(g, self.cams, T_cw, self.opts, self.rec, self.touched, self.jac, self.status, stream)

    def bin(self, stream=None) -> None:
        A.gs_bin_tiles(self.N, self.cams, self.opts, self.rec, self.touched, self.values, self.keys, self.ranges,
                       self.status, self.bin_ws, stream, order=self.order)

    def project_bin(self, g, T_cw: torch.Tensor, stream=None) -> None:
        """project() then bin() in one call, the projection counting the pairs
        (bit-identical outputs, one pass over the records fewer)."""
        A.gs_project_bin(g, self.cams, T_cw, self.opts, self.rec, self.touched, self.jac, self.values, self.keys,
                         self.ranges, self.status, self.bin_ws, stream, order=self.order)

    def forward(self, obs_depth: Optional[torch.Tensor] = None, stream=None) -> None:
        A.gs_render_fwd(self.N, self.cams, self.opts, self.rec, self.values, self.ranges, obs_depth, self.img,
                        self.status, stream, order=self.order, queue=self.queue)

    def backward(self, *, obs_depth=None, loss: Optional[dict] = None, dL: Optional[dict] = None,
                 g: Optional[Gaussians] = None, T_cw: Optional[torch.Tensor] = None, grads: Optional[dict] = None,
                 fused_pose: bool = True, stream=None) -> None:
        """Backward; with fused_pose the last CTA of each frame also writes
        ``pose_grad`` (otherwise call reduce_pose())."""
        A.gs_render_bwd(self.N, self.cams, self.opts, self.rec, self.jac, self.values, self.ranges, T_cw, g,
                        obs_depth, self.img, dL, loss, grads, self.pose_partials,
                        self.pose_grad if fused_pose else None, self.status, self.bwd_ws, stream, order=self.order,
                        queue=self.queue, touched=self.touched)

    def fwd_bwd_pose(self, loss: dict, images: bool = False, fused_pose: bool = True, stream=None,
                     adam_state=None, adam=None, T_cw=None) -> None:
        """Tracking pass (POSE mode): forward + backward of the colour/depth loss in
        one launch per tile; with images=True the tracking channels are written
        too (bit-identical to forward() + backward()); with adam_state (and adam,
        T_cw) the same launch also applies the pose Adam step."""
        out = {k: self.img[k] for k in ("color", "depth", "nu_map", "T_final", "n_last")} if images else None
        A.gs_render_fwd_bwd_pose(self.N, self.cams, self.opts, self.rec, self.jac, self.values, self.ranges, loss,
                                 out, self.pose_partials, self.pose_grad if fused_pose else None, self.status,
                                 self.bwd_ws, stream, order=self.order, adam_state=adam_state, adam=adam,
                                 T_cw=T_cw)

    def nu_accumulate(self, obs_depth: torch.Tensor, nu_num: torch.Tensor, nu_cnt: torch.Tensor,
                      dominant: Optional[torch.Tensor] = None, stream=None) -> None:
        """Eq. 13: add every dominated pixel of this batch's frames to nu_num
        (float64 [N]) and nu_cnt (int32 [N], used as uint32); needs a forward of a
        Rasterizer built with dominant=True."""
        if "dom_pos" not in self.img:
            raise ValueError("Rasterizer was built without dominant=True")
        A.gs_nu_accumulate(self.N, self.cams, self.rec, self.values, obs_depth, self.img, nu_num, nu_cnt, dominant,
                           self.status, stream)

    def estimate_nu(self, g: Gaussians, T_cw: torch.Tensor, obs_depth: torch.Tensor, tau: float = 0.025,
                    low_opacity: float = 0.01, dominant: Optional[torch.Tensor] = None) -> int:
        """Per-Gaussian uncertainty over this batch's keyframe window (Sec. 3.2):
        render, accumulate Eq. 13, set g.nu in place and lower the opacity of every
        Gaussian with nu > tau to ``low_opacity`` (tau <= 0: no opacity change).
        Returns how many Gaussians exceeded tau (synchronises)."""
        self.render(g, T_cw, obs_depth)
        num = torch.zeros(self.N, dtype=torch.float64, device=self.device)
        cnt = torch.zeros(self.N, dtype=torch.int32, device=self.device)
        n_over = torch.zeros(1, dtype=torch.int32, device=self.device)
        self.nu_accumulate(obs_depth, num, cnt, dominant)
        low = math.log(low_opacity / (1.0 - low_opacity))
        A.gs_nu_finalize(num, cnt, g.nu, tau, low, g.opacity_logit if tau > 0 else None, n_over, self.status)
        self.last_nu = (num, cnt)
        code, _ = self.read_status()
        if code != 0:
            raise A.GsError(code, "device status")
        return int(n_over.item())

    def reduce_pose(self, stream=None) -> None:
        A.gs_pose_grad_reduce(self.pose_partials, self.F, self.per_frame, self.pose_grad, self.status, stream)

    def render(self, g: Gaussians, T_cw: torch.Tensor, obs_depth=None, max_retries: int = 3) -> None:
        """project + bin + forward; grows the pair capacity and re-runs on overflow
        (reads the status word, i.e. synchronises)."""
        for _ in range(max_retries + 1):
            self.reset_status()
            self.project(g, T_cw)
            self.bin()
            self.forward(obs_depth)
            code, need = self.read_status()
            if code == 0:
                return
            if code != A.GS_ERR_CAPACITY:
                raise A.GsError(code, "device status")
            self.set_capacity(int(need * 1.25) + 1024)
        raise A.GsError(A.GS_ERR_CAPACITY, "pair capacity still exceeded")

    def step(self, g, T_cw: torch.Tensor, obs_depth=None, loss: Optional[dict] = None,
             grads: Optional[dict] = None, stream=None) -> None:
        """One batch step, enqueued without any host sync: project, bin,
        forward and, unless in FWD mode, the backward with the fused ``loss``
        (FULL mode: parameter gradients into ``grads``, overwritten)."""
        self.project(g, T_cw, stream)
        self.bin(stream)
        self.forward(obs_depth, stream)
        if self.mode == A.GS_MODE_FULL:
            self.backward(obs_depth=obs_depth, loss=loss, g=g, T_cw=T_cw, grads=grads, stream=stream)
        elif self.mode == A.GS_MODE_POSE:
            self.backward(obs_depth=obs_depth, loss=loss, stream=stream)

    def capture_step(self, g, T_cw: torch.Tensor, obs_depth=None, loss: Optional[dict] = None,
                     grads: Optional[dict] = None) -> "torch.cuda.CUDAGraph":
        """step() captured once in a CUDA graph on a side stream (after one
        eager run, which also raises the kernels' one-time attributes). The
        graph reads and writes the same tensors every replay: update their
        contents in place, then graph.replay(). Read the status word after a
        replay: a pair overflow needs set_capacity() and a new capture."""
        s = torch.cuda.Stream(device=self.device)
        s.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(s):
            self.step(g, T_cw, obs_depth, loss, grads, s)
        s.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=s):
            self.step(g, T_cw, obs_depth, loss, grads, s)
        return graph

    # --------------------------------------------------------------- views
    def frame_images(self, f: int) -> dict:
        """Per-frame views: color [3,H,W], the others [H,W]."""
        c = self.cams[f]
        H, W = int(c.height), int(c.width)
        off = sum(int(x.width) * int(x.height) for x in self.cams[:f])
        out = {"color": self.img["color"][3 * off: 3 * off + 3 * H * W].view(3, H, W)}
        for k in CHANNELS[1:] + ("dom_pos", "dom_weight"):
            if k in self.img:
                out[k] = self.img[k][off: off + H * W].view(H, W)
        return out

    def tile_lists(self):
        """(values[:P], ranges [n_tiles,2]) after a successful bin (synchronises)."""
        P = self.read_status()[1]
        return self.values[:P], self.ranges.view(-1, 2)


# ===================================================================== autotuner
_TUNE_CACHE: dict = {}


def autotune(cams: Sequence, g, T_cw: torch.Tensor, obs_depth=None, mode: int = A.GS_MODE_FULL,
             loss: Optional[dict] = None, tiles=(8, 16, 32), batches=(256, 512),
             scheds=(A.GS_SCHED_TILE, A.GS_SCHED_PERSISTENT), reps: int = 3, jclamp: float = 1.3,
             nu_cull: float = 0.0):
    """Picks the tile size (8, 16 or 32 pixels), the per-CTA staging batch of
    the blend kernels (256 or 512 list entries; 8x8 tiles always stage 64) and
    the schedule (one CTA per tile, or persistent CTAs pulling tiles from a
    device queue) of a frame batch, by timing one whole step (Rasterizer.step:
    project, bin, forward and, unless mode is FWD, the backward with the fused
    ``loss``) with CUDA events, ``reps`` times per candidate after one untimed
    run. Images and gradients do not depend on any of the three (same per-pixel
    lists and arithmetic), so the choice changes speed only. Results are cached
    per (resolutions, N, mode). Returns ((tile, batch, sched), {(tile, batch,
    sched): ms})."""
    key = (tuple((int(c.width), int(c.height)) for c in cams), int(g.n), int(mode), tuple(tiles), tuple(batches),
           tuple(scheds))
    if key in _TUNE_CACHE:
        return _TUNE_CACHE[key]
    full = mode == A.GS_MODE_FULL
    grads = {k: torch.empty_like(getattr(g, k)) for k in
             ("means", "log_scales", "quats", "opacity_logit", "colors", "nu")} if full else None
    times = {}
    cap = None
    for t in tiles:
        for b in (batches if t >= 16 else batches[:1]):  # 8x8 tiles stage 64 whatever the batch
            for sc in scheds:
                r = Rasterizer(cams, g.n, tile=t, mode=mode, jclamp=jclamp, nu_cull=nu_cull, batch=b, sched=sc)
                r.render(g, T_cw, obs_depth)
                r.set_capacity(int(r.read_status()[1] * 1.25) + 4096)
                r.step(g, T_cw, obs_depth, loss, grads)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(reps):
                    r.step(g, T_cw, obs_depth, loss, grads)
                e1.record()
                e1.synchronize()
                if r.read_status()[0] != 0:
                    raise A.GsError(r.read_status()[0], f"autotune tile {t} batch {b} sched {sc}")
                times[(t, b, sc)] = e0.elapsed_time(e1) / reps
                del r
    best = min(times, key=times.get)
    _TUNE_CACHE[key] = (best, times)
    return best, times


def autotune_tile(cams: Sequence, g, T_cw: torch.Tensor, obs_depth=None, mode: int = A.GS_MODE_FULL,
                  loss: Optional[dict] = None, candidates=(8, 16, 32), reps: int = 3, jclamp: float = 1.3,
                  nu_cull: float = 0.0):
    """autotune() over the tile size alone (batch 512, one CTA per tile).
    Returns (best tile, {tile: ms})."""
    best, times = autotune(cams, g, T_cw, obs_depth, mode, loss, tiles=candidates, batches=(512,),
                           scheds=(A.GS_SCHED_TILE,), reps=reps, jclamp=jclamp, nu_cull=nu_cull)
    return best[0], {k[0]: v for k, v in times.items()}


# ===================================================================== autograd
class GaussianRasterize(torch.autograd.Function):
    """Renders colour, depth, opacity, U, nu map and median depth of F frames at
    poses Exp(xi_f) T_cw_f (xi_f = 0 at the call) and differentiates w.r.t. every
    Gaussian parameter and xi (left se(3) perturbation, (rho, phi))."""

    @staticmethod
    def forward(ctx, means, log_scales, quats, opacity_logit, colors, nu, xi, T_cw, rast: Rasterizer,
                obs_depth=None):
        g = Gaussians(means.contiguous(), log_scales.contiguous(), quats.contiguous(),
                      opacity_logit.contiguous(), colors.contiguous(), nu.contiguous())
        T_cw = T_cw.contiguous()
        rast.render(g, T_cw, obs_depth)
        ctx.rast, ctx.g, ctx.T_cw, ctx.obs_depth = rast, g, T_cw, obs_depth
        im = rast.img
        outs = tuple(im[k].clone() for k in ("color", "depth", "alpha", "unc", "nu_map", "median"))
        return outs

    @staticmethod
    def backward(ctx, g_color, g_depth, g_alpha, g_unc, g_nu, g_median):
        rast: Rasterizer = ctx.rast
        g: Gaussians = ctx.g
        dL = {}
        for k, v in (("color", g_color), ("depth", g_depth), ("alpha", g_alpha), ("unc", g_unc), ("nu_map", g_nu),
                     ("median", g_median)):
            if v is not None:
                dL[k] = v.contiguous()
        if "unc" in dL and ctx.obs_depth is None:
            dL.pop("unc")
        dev = g.means.device
        grads = {k: torch.empty_like(getattr(g, k)) for k in
                 ("means", "log_scales", "quats", "opacity_logit", "colors", "nu")}
        rast.backward(obs_depth=ctx.obs_depth, dL=dL, g=g, T_cw=ctx.T_cw, grads=grads)
        code, _ = rast.read_status()
        if code:
            raise A.GsError(code, "device status in backward")
        gxi = rast.pose_grad.to(torch.float32).to(dev)
        return (grads["means"], grads["log_scales"], grads["quats"], grads["opacity_logit"], grads["colors"],
                grads["nu"], gxi, None, None, None)


def rasterize(g: Gaussians, xi: torch.Tensor, T_cw: torch.Tensor, rast: Rasterizer, obs_depth=None):
    """Differentiable render; returns dict of per-frame-concatenated channels."""
    outs = GaussianRasterize.apply(g.means, g.log_scales, g.quats, g.opacity_logit, g.colors, g.nu, xi, T_cw,
                                   rast, obs_depth)
    return dict(zip(("color", "depth", "alpha", "unc", "nu_map", "median"), outs))


# ===================================================================== tracking
def pose_state(T: torch.Tensor) -> torch.Tensor:
    """FP64 pose state [F, 28]: R (9), t (3), Adam m (6), v (6), step,
    beta1^step, beta2^step, unused."""
    T = T.reshape(-1, 3, 4).to(torch.float64)
    st = torch.zeros(T.shape[0], A.GS_POSE_STATE_DOUBLES, dtype=torch.float64, device=T.device)
    st[:, :9] = T[:, :, :3].reshape(-1, 9)
    st[:, 9:12] = T[:, :, 3]
    st[:, 25:27] = 1.0
    return st


def state_pose(st: torch.Tensor) -> torch.Tensor:
    T = torch.zeros(st.shape[0], 3, 4, dtype=torch.float64, device=st.device)
    T[:, :, :3] = st[:, :9].view(-1, 3, 3)
    T[:, :, 3] = st[:, 9:12]
    return T


class Tracker:
    """Sequential tracking (Sec. 3.4, Eq. 19-20) of one frame: ``iters``
    iterations of project -> bin -> forward -> POSE backward with the fused
    uncertainty-weighted L1 colour + depth loss -> FP64 pose reduction -> Adam
    step on the pose, all on the device. With ``graph=True`` one iteration is
    captured once in a CUDA graph and replayed."""

    def __init__(self, g, cam, tile: int = 16, iters: int = 30, lam=(0.2, 1.0), unc_tau: float = 0.025,
                 lr_rot: float = 0.0015, lr_trans: float = 0.00215, jclamp: float = 1.3, graph: bool = True,
                 capacity: Optional[int] = None, timing: bool = False, fused: bool = True,
                 timing_every: int = 1):
        self.g = g
        self.cam = cam
        self.iters = iters
        self.graph_enabled = graph
        # fused: forward and backward in one launch per tile (gs_render_fwd_bwd_pose);
        # otherwise gs_render_fwd then gs_render_bwd (same results, bit for bit)
        self.fused = fused
        # optional per-iteration CUDA events around each backward launch (recorded
        # inside the captured graph as event nodes), for per-kernel timing; with
        # timing_every = k only iterations 0, k, 2k, ... carry them (each pair of
        # event nodes costs ~9 us of an iteration: it also breaks the kernel-to-
        # kernel launch chaining around the timed launch)
        self.timing = timing
        self.timing_every = max(1, int(timing_every))
        self.bwd_events = ([(torch.cuda.Event(enable_timing=True, external=True),
                             torch.cuda.Event(enable_timing=True, external=True))
                            if it % self.timing_every == 0 else None for it in range(iters)]
                           if timing else None)
        dev = (g.packed if isinstance(g, PackedGaussians) else g.means).device
        self.rast = Rasterizer([cam], g.n, tile=tile, mode=A.GS_MODE_POSE, capacity=capacity, jclamp=jclamp,
                               channels="track")
        H, W = int(cam.height), int(cam.width)
        self.target_color = torch.zeros(3 * H * W, dtype=torch.float32, device=dev)
        self.target_depth = torch.zeros(H * W, dtype=torch.float32, device=dev)
        self.loss = dict(w_color=lam[0], w_depth=lam[1], w_unc=0.0, w_nu=0.0, unc_tau=unc_tau,
                         target_color=self.target_color, target_depth=self.target_depth)
        self.adam = A.gs_adam(lr_rot, lr_trans, 0.9, 0.999, 1e-8)
        self.state = torch.zeros(1, A.GS_POSE_STATE_DOUBLES, dtype=torch.float64, device=dev)
        self.T_cw = torch.zeros(12, dtype=torch.float32, device=dev)
        self.stream = torch.cuda.Stream(device=dev)
        self.graph = None

    # one iteration, enqueued on `stream`
    def _iteration(self, stream=None, it: int = 0):
        r = self.rast
        r.project_bin(self.g, self.T_cw, stream)
        ev = self.bwd_events[it] if self.bwd_events is not None else None
        if self.fused:  # forward, backward, pose reduction and Adam step in one launch
            if ev:
                ev[0].record(stream)
            r.fwd_bwd_pose(self.loss, stream=stream, adam_state=self.state, adam=self.adam, T_cw=self.T_cw)
            if ev:
                ev[1].record(stream)
        else:
            r.forward(self.target_depth, stream)
            if ev:
                ev[0].record(stream)
            r.backward(obs_depth=self.target_depth, loss=self.loss, stream=stream)  # + fused pose reduction
            if ev:
                ev[1].record(stream)
            A.gs_pose_adam_step(self.state, r.pose_grad, self.T_cw, 1, self.adam, r.status, stream)

    def kernel_launches_per_iteration(self) -> int:
        """libgs kernels one iteration launches: the tile-counter clear, the
        projection (which also counts the pairs), the tile scan, fill and
        per-tile sort; then either the tracking pass (forward and backward in
        one launch) and the pose reduction with the Adam step (one chained
        launch), or the forward, the backward (with the pose reduction) and
        the Adam step. No memsets."""
        return 5 + (2 if self.fused else 3)

    def _capture(self):
        """Capture all ``iters`` iterations of a frame in one CUDA graph."""
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(self.stream):
            self._iteration(self.stream)  # warm-up outside capture
        self.stream.synchronize()
        with torch.cuda.graph(self.graph, stream=self.stream):
            for it in range(self.iters):
                self._iteration(self.stream, it)

    def backward_ms(self) -> list:
        """Per-iteration duration of the backward launch in the last frame (the
        fused forward + backward launch when fused; needs timing=True and a
        completed frame)."""
        return [e[0].elapsed_time(e[1]) for e in self.bwd_events if e is not None]

    def stage_ms(self, target_color, target_depth, T_init) -> dict:
        """Mean device time per iteration of each library call of a tracking
        iteration, over one frame captured in a CUDA graph with an event node
        around every call (events break the kernel-to-kernel chaining, so the
        stages add up to a little more than an iteration of the plain graph):
        "project_bin" (counter clear, projection with pair count, tile scan,
        fill and sort) and "tracking_pass" (the pass, then the pose reduction
        with the Adam step; fused=False: forward, backward and Adam)."""
        marks = [[torch.cuda.Event(enable_timing=True, external=True) for _ in range(3)]
                 for _ in range(self.iters)]
        r, s = self.rast, self.stream
        self.set_frame(target_color, target_depth, T_init)
        s.wait_stream(torch.cuda.current_stream())
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=s):
            for e in marks:
                e[0].record(s)
                r.project_bin(self.g, self.T_cw, s)
                e[1].record(s)
                if self.fused:
                    r.fwd_bwd_pose(self.loss, stream=s, adam_state=self.state, adam=self.adam, T_cw=self.T_cw)
                else:
                    r.forward(self.target_depth, s)
                    r.backward(obs_depth=self.target_depth, loss=self.loss, stream=s)
                    A.gs_pose_adam_step(self.state, r.pose_grad, self.T_cw, 1, self.adam, r.status, s)
                e[2].record(s)
        self.set_frame(target_color, target_depth, T_init)
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            graph.replay()
        s.synchronize()
        n = len(marks)
        return {"project_bin": sum(e[0].elapsed_time(e[1]) for e in marks) / n,
                "tracking_pass": sum(e[1].elapsed_time(e[2]) for e in marks) / n}

    def set_frame(self, target_color: torch.Tensor, target_depth: torch.Tensor, T_init: torch.Tensor) -> None:
        self.target_color.copy_(target_color.reshape(-1), non_blocking=True)
        self.target_depth.copy_(target_depth.reshape(-1), non_blocking=True)
        st = pose_state(T_init.to(self.state.device))
        self.state.copy_(st)
        self.T_cw.copy_(state_pose(st).reshape(-1).to(torch.float32))
        self.rast.status.zero_()

    def run(self) -> None:
        """Enqueue ``iters`` iterations on the tracker's stream (no host sync)."""
        cur = torch.cuda.current_stream()
        self.stream.wait_stream(cur)
        with torch.cuda.stream(self.stream):
            if self.graph is not None:
                self.graph.replay()
            else:
                for it in range(self.iters):
                    self._iteration(self.stream, it)
        cur.wait_stream(self.stream)

    def track_host(self, target_color, target_depth, T_init, out=None) -> torch.Tensor:
        """End-to-end call with host buffers: copies the frame's RGB-D target and
        initial pose (pinned host tensors) to the device, tracks, and copies the
        refined pose (FP64 [3,4]) back to ``out`` (pinned host) or a new tensor."""
        dev = self.state.device
        tc = target_color.to(dev, non_blocking=True)
        td = target_depth.to(dev, non_blocking=True)
        T0 = T_init.to(dev, non_blocking=True)
        T = self.track(tc, td, T0)
        if out is None:
            return T.cpu()
        out.copy_(T, non_blocking=True)
        torch.cuda.current_stream().synchronize()
        return out

    # ------------------------------------------------------------ streaming
    def submit(self, target_color, target_depth, T_init, out) -> None:
        """Enqueue one frame from pinned host memory and return at once.

        The frame's RGB-D target and initial pose (pinned host tensors) are
        copied on a separate copy stream into one of two device staging
        buffers, so the upload of frame k + 1 overlaps the tracking of frame k.
        The frame is then set and tracked in stream order after everything
        already enqueued on the caller's current stream. Its refined pose
        (FP64 [3, 4]) is copied to ``out`` (pinned host) and its status word to
        an internal pinned slot, both without a host sync. The host tensors
        must stay untouched until drain() returns. Needs a captured graph
        (prepare() or one track()/track_host() call first)."""
        if self.graph_enabled and self.graph is None:
            raise RuntimeError("submit() needs the graph captured: call prepare() or track() once first")
        dev = self.state.device
        if not hasattr(self, "_copy_stream"):
            self._copy_stream = torch.cuda.Stream(device=dev)
            self._stage = [(torch.empty_like(self.target_color), torch.empty_like(self.target_depth),
                            torch.empty(3, 4, dtype=torch.float64, device=dev)) for _ in range(2)]
            self._staged = [torch.cuda.Event() for _ in range(2)]
            self._consumed = [torch.cuda.Event() for _ in range(2)]
            self._pending = []
        k = len(self._pending)
        slot = k % 2
        col, dep, T0 = self._stage[slot]
        cur = torch.cuda.current_stream()
        with torch.cuda.stream(self._copy_stream):
            if k >= 2:  # the slot's previous frame has been copied out of it
                self._copy_stream.wait_event(self._consumed[slot])
            col.copy_(target_color.reshape(-1), non_blocking=True)
            dep.copy_(target_depth.reshape(-1), non_blocking=True)
            T0.copy_(T_init.reshape(3, 4), non_blocking=True)
            self._staged[slot].record(self._copy_stream)
        cur.wait_event(self._staged[slot])
        self.set_frame(col, dep, T0)
        self._consumed[slot].record(cur)
        self.run()
        status = torch.empty(2, dtype=torch.int32).pin_memory()
        out.copy_(state_pose(self.state)[0], non_blocking=True)
        status.copy_(self.rast.status[:2], non_blocking=True)
        self._pending.append((target_color, target_depth, T_init, out, status))

    def drain(self, max_retries: int = 3) -> int:
        """Wait for every submitted frame; a frame whose pair buffer overflowed
        is tracked again (synchronously, with a larger buffer) into its
        ``out``. Returns the number of frames completed; raises GsError for any
        other device status."""
        torch.cuda.current_stream().synchronize()
        pending, self._pending = getattr(self, "_pending", []), []
        for color, depth, T_init, out, status in pending:
            code = int(status[0])
            if code == A.GS_ERR_CAPACITY:
                self.track_host(color, depth, T_init, out)
            elif code != 0:
                raise A.GsError(code, "device status during tracking")
        return len(pending)

    def track(self, target_color, target_depth, T_init, max_retries: int = 3) -> torch.Tensor:
        """Track one frame; returns the refined pose [3,4] (FP64, on device).
        Grows the pair capacity (and re-captures the graph) on overflow."""
        for _ in range(max_retries + 1):
            self.set_frame(target_color, target_depth, T_init)
            if self.graph_enabled and self.graph is None:
                self._capture()
                self.set_frame(target_color, target_depth, T_init)
            self.run()
            code, need = self.rast.read_status()
            if code == 0:
                return state_pose(self.state)[0]
            if code != A.GS_ERR_CAPACITY:
                raise A.GsError(code, "device status during tracking")
            self.rast.set_capacity(int(need * 1.5) + 4096)
            self.graph = None
        raise A.GsError(A.GS_ERR_CAPACITY, "pair capacity still exceeded")

    def prepare(self, target_color, target_depth, T_init, headroom: float = 1.5) -> None:
        """Size the pair buffer from one render at T_init (with headroom), then
        capture the graph."""
        self.set_frame(target_color, target_depth, T_init)
        self.rast.render(self.g, self.T_cw, self.target_depth)
        need = self.rast.read_status()[1]
        self.rast.set_capacity(int(need * headroom) + 4096)
        self.graph = None
        if self.graph_enabled:
            self.set_frame(target_color, target_depth, T_init)
            self._capture()
