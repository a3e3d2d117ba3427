"""B300 (sm_103a) differentiable tile-based 3D Gaussian rasterizer of CG-SLAM
(arXiv 2403.16095): EWA projection, 64-bit-key radix tile binning, front-to-back
blending of colour / depth / opacity / depth uncertainty, and a reverse-walk
backward to every Gaussian parameter and to the se(3) camera pose.

The compute lives in libgs.so (C ABI, include/gs.h); this package is its thin
Python binding (``_abi``) plus a PyTorch-side driver (``raster``). Importing it
loads libgs.so and fails loudly if the library has not been built.
"""
from . import _abi  # noqa: F401  (loads libgs.so)
from ._abi import GsError, Gaussians  # noqa: F401
from .raster import GaussianRasterize, Rasterizer, Tracker, rasterize  # noqa: F401

__all__ = ["GsError", "Gaussians", "GaussianRasterize", "Rasterizer", "Tracker", "rasterize"]
