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
    dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)
    off = 0
    for k in keys:
        n = grads[k].numel()
        grads[k].copy_(flat[off:off + n].view_as(grads[k]))
        off += n
    return grads
