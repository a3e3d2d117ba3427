"""Writes tests/golden/tiny_oracle.json from the FP64 oracle alone.

The paper (arXiv 2403.16095) prints no worked numeric example of the
rasterizer, so the stored values here are a regression fixture of the oracle
on the seeded 128x96 / 2,000-Gaussian scene: sampled pixels of every rendered
channel (Eq. 3-10), the loss (Eq. 14/16/19 with the optional |U| and nu terms)
and the left se(3) pose gradient (Sec. 3.4). Run from the repository root:
    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

PIX = [0, 77, 1500, 6143, 6208, 7001, 9999, 12287]


def compute():
    sc, cam, T = synth.tiny_scene()
    tc, td = synth.random_targets(cam, 1001 + 70)
    im = oracle.render(sc, cam, T, obs_depth=td[0])
    L = oracle.LossSpec(1.0, 1.0, 1.0, 1.0, 0.0, tc[0], td[0])
    g = oracle.grad(sc, cam, T, L)
    out = {"pixels": PIX}
    for k in ("depth", "alpha", "unc", "nu_map", "median", "T_final"):
        out[k] = [float(v) for v in im[k].reshape(-1)[PIX]]
    out["color"] = [[float(v) for v in im["color"].reshape(3, -1)[:, p]] for p in PIX]
    out["n_contrib"] = [int(v) for v in im["n_contrib"].reshape(-1)[PIX]]
    out["loss"] = float(g["loss"])
    out["pose_grad"] = [float(v) for v in g["pose"]]
    return out


if __name__ == "__main__":
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tiny_oracle.json")
    with open(path, "w") as f:
        json.dump(compute(), f, indent=1)
    print("wrote", path)
