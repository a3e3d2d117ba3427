"""B300 (sm_103a) differentiable tile-based 3D Gaussian rasterizer of CG-SLAM
(arXiv 2403.16095): EWA projection, 64-bit-key radix tile binning, front-to-back
blending of colour / depth / opacity / depth uncertainty, and a reverse-walk
backward to every Gaussian parameter and to the se(3) camera pose.

The compute lives in libgs.so (C ABI, include/gs.h); this package is its thin
Python binding (``_abi``) plus PyTorch-side host code (``raster``). The public
names load libgs.so on first use and fail loudly if it has not been built
(``python -m paper_2403_16095_b300.build``); importing the package alone does
not, so the build step never depends on an earlier build.
"""
import importlib

_EXPORTS = {
    "GsError": "_abi", "Gaussians": "_abi", "PackedGaussians": "_abi", "pack_bf16": "_abi",
    "GaussianRasterize": "raster", "Rasterizer": "raster", "Tracker": "raster", "rasterize": "raster",
    "autotune_tile": "raster", "autotune": "raster",
}

__all__ = sorted(_EXPORTS)


def __getattr__(name):
    if name in ("_abi", "raster"):
        return importlib.import_module(f".{name}", __name__)
    if name in _EXPORTS:
        return getattr(importlib.import_module(f".{_EXPORTS[name]}", __name__), name)
    raise AttributeError(name)
