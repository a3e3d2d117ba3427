"""Helpers shared by the GPU parity tests (inputs come from synth/, expected
values from oracle/; nothing here computes rasterizer arithmetic)."""
import numpy as np
import torch

PARAMS = ("means", "log_scales", "quats", "opacity_logit", "colors", "nu")


def to_gpu_gaussians(sc):
    from paper_2403_16095_b300 import Gaussians
    return Gaussians(*(torch.from_numpy(np.ascontiguousarray(np.asarray(getattr(sc, k), np.float32))).cuda()
                       for k in PARAMS))


def f32_scene(sc):
    """The FP32 values the GPU sees, widened back to FP64 for the oracle."""
    import synth
    return synth.Scene(*(np.asarray(np.asarray(getattr(sc, k), np.float32), np.float64) for k in PARAMS))


def poses_gpu(T):
    T = np.asarray(T, np.float32).reshape(-1, 3, 4)
    return torch.from_numpy(np.ascontiguousarray(T)).cuda().reshape(-1)


def rec_fields(r):
    """Decode the packed projection records of a Rasterizer into numpy arrays."""
    rec = r.rec.view(-1, 16).cpu()
    f = rec.numpy()
    rect = rec.view(torch.int32).numpy()[:, 12:16]
    return dict(mean2d=f[:, 0:2], conic=f[:, 2:5], opacity=f[:, 5], depth=f[:, 6], nu=f[:, 7],
                color=f[:, 8:11], radius=f[:, 11], rect=rect, valid=rect[:, 0] <= rect[:, 2])


def decision_margin(ora, pix_mask=None):
    """Per-pixel minimum of the oracle's normalised decision margins."""
    m = ora["margins"].min(axis=0)
    return m if pix_mask is None else m[pix_mask]
