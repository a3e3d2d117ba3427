"""Frame sharding of a keyframe window across ranks (one process per GPU).

Mapping renders and differentiates whole keyframes (the window of Eq. 21).
Frames are independent up to the final per-Gaussian gradient, which is a sum
over frames; so each rank takes whole frames, runs the FULL backward on them
with the replicated Gaussian field, and one SUM all-reduce of the flattened
parameter gradients is the only exchange. Per-frame pose gradients stay with
the rank that owns the frame. Tracking (one frame's iterations depend on each
other) does not shard: it runs as independent replicas.
"""
from typing import Dict, List, Optional, Sequence

import numpy as np

import torch
import torch.distributed as dist


def frames_for_rank(n_frames: int, rank: int, world: int) -> List[int]:
    """Round-robin assignment: frame f belongs to rank f mod world. Every frame
    lands on exactly one rank; ranks differ by at most one frame."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside world of size {world}")
    if n_frames < 0:
        raise ValueError("n_frames must be non-negative")
    return list(range(rank, n_frames, world))


def allreduce_gaussian_grads(grads: Dict[str, torch.Tensor], names: Optional[Sequence[str]] = None,
                             group=None) -> Dict[str, torch.Tensor]:
    """Sum the per-Gaussian gradients over ranks in one collective.

    The tensors are packed into one contiguous buffer (in ``names`` order, else
    sorted key order, identical on every rank), summed with a single all-reduce
    and unpacked in place. A world of one returns the input untouched."""
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size(group) == 1:
        return grads
    keys = list(names) if names is not None else sorted(grads)
    flat = torch.cat([grads[k].reshape(-1) for k in keys])
    if flat.is_cuda and dist.get_backend(group) == "gloo":
        # gloo reduces host memory: stage the packed buffer through the host
        host = flat.cpu()
        dist.all_reduce(host, op=dist.ReduceOp.SUM, group=group)
        flat.copy_(host)
    else:
        dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)
    off = 0
    for k in keys:
        n = grads[k].numel()
        grads[k].copy_(flat[off:off + n].view_as(grads[k]))
        off += n
    return grads


PARAMS = ("means", "log_scales", "quats", "opacity_logit", "colors", "nu")


def window_slice(cams, T_cw, target_color, target_depth, frames: Sequence[int]):
    """The cameras, poses ([F*12]) and RGB-D targets of the listed frames of a
    window, in that order. The window's images are planar and concatenated
    frame after frame (colour [3][H_f][W_f] per frame), so frames of different
    sizes are sliced by their pixel offsets."""
    frames = list(frames)
    T = T_cw.reshape(len(cams), 12)
    sizes = [int(c.width) * int(c.height) for c in cams]
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    tc = target_color.reshape(-1)
    td = target_depth.reshape(-1)
    if not frames:
        return [], T[:0].reshape(-1), tc[:0], td[:0]
    return ([cams[f] for f in frames], T[frames].contiguous().reshape(-1),
            torch.cat([tc[3 * offs[f]: 3 * offs[f + 1]] for f in frames]),
            torch.cat([td[offs[f]: offs[f + 1]] for f in frames]))


class ShardedWindow:
    """One rank's share of a keyframe window (Eq. 21): the frames
    ``frames_for_rank(len(cams), rank, world)`` of the window, rendered and
    differentiated (FULL mode, fused loss of Eq. 14, 16, 11, 12) in one launch
    per stage, then one SUM all-reduce of the per-Gaussian parameter gradients.
    The Gaussian field is replicated on every rank; pose gradients stay with the
    rank that owns the frame.

    cams / T_cw / targets describe the WHOLE window; each rank keeps its own
    frames' slices. T_cw: [F, 3, 4] (or [F*12]) FP32 on this rank's device;
    target_color [F, 3, H, W] and target_depth [F, H, W] (the sensor depth of U)
    on the device, every frame of the window the same size or not."""

    def __init__(self, cams, n_gaussians: int, T_cw, target_color, target_depth, rank: int = 0, world: int = 1,
                 tile: int = 16, loss_weights: Optional[dict] = None, group=None, capacity: Optional[int] = None,
                 batch: int = 0, sched: int = 0):
        from . import _abi as A
        from .raster import Rasterizer
        self.frames = frames_for_rank(len(cams), rank, world)
        self.rank, self.world, self.group = rank, world, group
        self.cams, self.T_cw, self.target_color, self.target_depth = window_slice(
            cams, T_cw, target_color, target_depth, self.frames)
        w = dict(w_color=0.7, w_depth=0.25, w_unc=0.15, w_align=0.25) if loss_weights is None else dict(loss_weights)
        self.loss = dict(w, target_color=self.target_color, target_depth=self.target_depth)
        self.rast = (Rasterizer(self.cams, n_gaussians, tile=tile, mode=A.GS_MODE_FULL, capacity=capacity,
                                batch=batch, sched=sched) if self.frames else None)

    def prepare(self, g) -> None:
        """One render to size the pair buffer (synchronises)."""
        if self.rast is not None:
            self.rast.render(g, self.T_cw, self.target_depth)
            self.rast.set_capacity(int(self.rast.read_status()[1] * 1.25) + 4096)

    def step(self, g, grads: Dict[str, torch.Tensor], allreduce: bool = True) -> None:
        """project, bin, forward and FULL backward of this rank's frames into
        ``grads`` (overwritten), then the gradient all-reduce over the ranks. No
        host synchronisation besides the collective."""
        if self.rast is not None:
            r = self.rast
            r.project(g, self.T_cw)
            r.bin()
            r.forward(self.target_depth)
            r.backward(obs_depth=self.target_depth, loss=self.loss, g=g, T_cw=self.T_cw, grads=grads)
        else:
            for k in PARAMS:
                grads[k].zero_()
        if allreduce:
            allreduce_gaussian_grads(grads, PARAMS, self.group)

    def pose_grads(self) -> Dict[int, torch.Tensor]:
        """FP64 se(3) gradient (rho, phi) of each frame this rank owns."""
        if self.rast is None:
            return {}
        return {f: self.rast.pose_grad[i] for i, f in enumerate(self.frames)}

    def status(self):
        return (0, 0) if self.rast is None else self.rast.read_status()
