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


# One image tolerance and one decision margin for every GPU-vs-oracle image
# comparison (the derivation is in the design notes, "FP32/FP64 decision flips"):
#   IMG_TOL          absolute, on every rendered channel: colour, depth, opacity,
#                    U, nu map, T_final, median depth;
#   DECISION_MARGIN  relative oracle margin of a threshold decision below which
#                    FP32 and FP64 may decide differently: q vs 9, alpha vs 1/255,
#                    T' vs 1e-4, opacity*G vs 0.99, T vs 0.5 (median), and the lead
#                    of the largest blend weight (dominant entry, Eq. 13). FP32
#                    carries T through up to a few hundred multiplications (~n 2^-24
#                    relative) and q through a cancelling sum of three terms;
#   ORDER_MARGIN     relative depth gap of neighbouring list entries below which the
#                    FP32 z order may differ from the FP64 one.
IMG_TOL = 1e-4
DECISION_MARGIN = 1e-4
ORDER_MARGIN = 1e-5
CHANNELS = ("color", "depth", "alpha", "unc", "nu_map", "T_final", "median")


def at_decision_margin(ora):
    """Per pixel (or sample): True where some oracle decision sits within the
    margins above, i.e. where FP32 may legitimately take another branch."""
    m = ora["margins"]
    return (m[[0, 1, 2, 3, 5]].min(axis=0) < DECISION_MARGIN) | (m[4] < ORDER_MARGIN)


def image_mismatch(im, ora, channels=CHANNELS, pix=None):
    """Per pixel: some channel differs from the oracle by more than IMG_TOL.
    im: GPU images ([3,H,W] colour, [H,W] others); ora: oracle images, full
    ([..,H,W]) or sampled at the flat pixel indices ``pix`` ([..,n])."""
    bad = None
    for k in channels:
        if k not in im or k not in ora:
            continue
        got = np.asarray(im[k])
        want = ora[k]
        if pix is not None:
            got = got.reshape(3, -1)[:, pix] if k == "color" else got.reshape(-1)[pix]
        e = np.abs(got - want)
        if k == "color":
            e = e.max(0)
        bad = e > IMG_TOL if bad is None else bad | (e > IMG_TOL)
    return bad
