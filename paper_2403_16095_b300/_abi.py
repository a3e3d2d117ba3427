"""ctypes binding of libgs (include/gs.h): argument marshalling only.

Each public function has the name of the C entry point it calls and takes
torch tensors (device memory) plus small Python/ctypes structs; it checks
dtype, device, contiguity and size, passes raw pointers through, and raises
``GsError`` with ``gs_last_error()`` if the call returns a non-OK status.
There is no fallback: if libgs.so is missing the import fails loudly.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Optional, Sequence

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libgs.so")

GS_MAX_FRAMES = 64
GS_REC_FLOATS = 16
GS_JAC_FLOATS = 36
GS_POSE_STATE_DOUBLES = 28
GS_MODE_FWD, GS_MODE_POSE, GS_MODE_FULL = 0, 1, 2
GS_SCHED_TILE, GS_SCHED_PERSISTENT = 0, 1
GS_OK, GS_ERR_INVALID_ARG, GS_ERR_CAPACITY, GS_ERR_CUDA, GS_ERR_TIMEOUT, GS_ERR_UNSUPPORTED = range(6)
STATUS_NAMES = {0: "GS_OK", 1: "GS_ERR_INVALID_ARG", 2: "GS_ERR_CAPACITY", 3: "GS_ERR_CUDA",
                4: "GS_ERR_TIMEOUT", 5: "GS_ERR_UNSUPPORTED"}


class GsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_fp = C.POINTER(C.c_float)
_dp = C.POINTER(C.c_double)
_vp = C.c_void_p


class gs_camera(C.Structure):
    _fields_ = [("width", C.c_int), ("height", C.c_int), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("znear", C.c_float)]


class gs_gaussians(C.Structure):
    _fields_ = [("n", C.c_int), ("means", _vp), ("log_scales", _vp), ("quats", _vp),
                ("opacity_logit", _vp), ("colors", _vp), ("nu", _vp)]


class gs_opts(C.Structure):
    _fields_ = [("tile", C.c_int), ("mode", C.c_int), ("jclamp", C.c_float), ("nu_cull", C.c_float),
                ("batch", C.c_int), ("sched", C.c_int)]


class gs_projected(C.Structure):
    _fields_ = [("n_gaussians", C.c_int), ("n_frames", C.c_int), ("rec", _vp), ("tiles_touched", _vp),
                ("pose_jac", _vp)]


class gs_tiles(C.Structure):
    _fields_ = [("capacity", C.c_int), ("n_tiles", C.c_int), ("values", _vp), ("keys", _vp), ("ranges", _vp),
                ("order", _vp), ("queue", _vp)]


class gs_image(C.Structure):
    _fields_ = [("color", _vp), ("depth", _vp), ("alpha", _vp), ("unc", _vp), ("nu_map", _vp),
                ("median", _vp), ("T_final", _vp), ("n_last", _vp), ("n_contrib", _vp), ("median_pos", _vp),
                ("dom_pos", _vp), ("dom_weight", _vp)]


class gs_image_grad(C.Structure):
    _fields_ = [("color", _vp), ("depth", _vp), ("alpha", _vp), ("unc", _vp), ("nu_map", _vp), ("median", _vp)]


class gs_loss(C.Structure):
    _fields_ = [("w_color", C.c_float), ("w_depth", C.c_float), ("w_unc", C.c_float), ("w_nu", C.c_float),
                ("unc_tau", C.c_float), ("target_color", _vp), ("target_depth", _vp), ("w_align", C.c_float)]


class gs_gaussians_bf16(C.Structure):
    _fields_ = [("n", C.c_int), ("anchors", _vp), ("packed", _vp)]


GS_BF16_CHUNK = 256


class gs_grads(C.Structure):
    _fields_ = [("means", _vp), ("log_scales", _vp), ("quats", _vp), ("opacity_logit", _vp),
                ("colors", _vp), ("nu", _vp)]


class gs_adam(C.Structure):
    _fields_ = [("lr_rot", C.c_float), ("lr_trans", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float),
                ("eps", C.c_float)]


EXPORTS = ("gs_abi_version", "gs_last_error", "gs_project", "gs_bin_tiles_workspace_size", "gs_bin_tiles",
           "gs_bin_tiles_noalloc", "gs_render_fwd", "gs_pose_partials_per_frame", "gs_render_bwd_workspace_size",
           "gs_render_bwd", "gs_render_fwd_bwd_pose", "gs_project_bf16", "gs_spatial_order_workspace_size", "gs_spatial_order",
           "gs_pack_bf16", "gs_nu_accumulate", "gs_nu_finalize", "gs_pose_grad_reduce", "gs_pose_adam_step",
           "gs_project_bin", "gs_project_bin_bf16")
GS_NOALLOC_MAX_PAIRS = 1 << 19
ABI_VERSION = 9  # GS_ABI_VERSION of the gs.h these structures mirror


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libgs.so not built at {LIB_PATH}; run `python -m paper_2403_16095_b300.build`")
    lib = C.CDLL(LIB_PATH)
    lib.gs_abi_version.restype = C.c_int
    if lib.gs_abi_version() != ABI_VERSION:
        raise ImportError(f"libgs.so has ABI {lib.gs_abi_version()}, this binding needs {ABI_VERSION}; rebuild it")
    lib.gs_last_error.restype = C.c_char_p
    lib.gs_project.argtypes = [C.POINTER(gs_gaussians), C.c_int, C.POINTER(gs_camera), _vp,
                               C.POINTER(gs_opts), C.POINTER(gs_projected), _vp, _vp]
    lib.gs_project_bf16.argtypes = [C.POINTER(gs_gaussians_bf16), C.c_int, C.POINTER(gs_camera), _vp,
                                    C.POINTER(gs_opts), C.POINTER(gs_projected), _vp, _vp]
    lib.gs_spatial_order_workspace_size.argtypes = [C.c_int]
    lib.gs_spatial_order_workspace_size.restype = C.c_size_t
    lib.gs_spatial_order.argtypes = [_vp, C.c_int, _vp, _vp, C.c_size_t, _vp, _vp]
    lib.gs_pack_bf16.argtypes = [C.POINTER(gs_gaussians), _vp, _vp, _vp, _vp, _vp]
    lib.gs_bin_tiles_workspace_size.argtypes = [C.c_int, C.c_int]
    lib.gs_bin_tiles_workspace_size.restype = C.c_size_t
    lib.gs_bin_tiles.argtypes = [C.POINTER(gs_projected), C.c_int, C.POINTER(gs_camera), C.POINTER(gs_opts),
                                 C.POINTER(gs_tiles), _vp, _vp, C.c_size_t, _vp]
    lib.gs_project_bin.argtypes = [C.POINTER(gs_gaussians), C.c_int, C.POINTER(gs_camera), _vp,
                                   C.POINTER(gs_opts), C.POINTER(gs_projected), C.POINTER(gs_tiles), _vp, _vp,
                                   C.c_size_t, _vp]
    lib.gs_project_bin_bf16.argtypes = [C.POINTER(gs_gaussians_bf16), C.c_int, C.POINTER(gs_camera), _vp,
                                        C.POINTER(gs_opts), C.POINTER(gs_projected), C.POINTER(gs_tiles), _vp, _vp,
                                        C.c_size_t, _vp]
    lib.gs_bin_tiles_noalloc.argtypes = [C.POINTER(gs_projected), C.c_int, C.POINTER(gs_camera),
                                         C.POINTER(gs_opts), C.POINTER(gs_tiles), _vp, _vp]
    lib.gs_bin_tiles_noalloc.restype = C.c_int
    lib.gs_render_fwd.argtypes = [C.POINTER(gs_projected), C.POINTER(gs_tiles), C.c_int, C.POINTER(gs_camera),
                                  _vp, C.POINTER(gs_opts), C.POINTER(gs_image), _vp, _vp]
    lib.gs_pose_partials_per_frame.argtypes = [C.c_int, C.c_int, C.c_int, C.POINTER(gs_camera), C.c_int]
    lib.gs_pose_partials_per_frame.restype = C.c_int
    lib.gs_render_bwd_workspace_size.argtypes = [C.c_int, C.c_int]
    lib.gs_render_bwd_workspace_size.restype = C.c_size_t
    lib.gs_render_bwd.argtypes = [C.POINTER(gs_projected), C.POINTER(gs_tiles), C.c_int, C.POINTER(gs_camera),
                                  _vp, C.POINTER(gs_gaussians), _vp, C.POINTER(gs_image),
                                  C.POINTER(gs_image_grad), C.POINTER(gs_loss), C.POINTER(gs_opts),
                                  C.POINTER(gs_grads), _vp, _vp, _vp, _vp, C.c_size_t, _vp]
    lib.gs_render_fwd_bwd_pose.argtypes = [C.POINTER(gs_projected), C.POINTER(gs_tiles), C.c_int,
                                           C.POINTER(gs_camera), C.POINTER(gs_loss), C.POINTER(gs_opts),
                                           C.POINTER(gs_image), _vp, _vp, _vp, C.POINTER(gs_adam), _vp, _vp, _vp,
                                           C.c_size_t, _vp]
    lib.gs_nu_accumulate.argtypes = [C.POINTER(gs_projected), C.POINTER(gs_tiles), C.c_int, C.POINTER(gs_camera),
                                     _vp, C.POINTER(gs_image), _vp, _vp, _vp, _vp, _vp]
    lib.gs_nu_finalize.argtypes = [C.c_int, _vp, _vp, _vp, C.c_float, C.c_float, _vp, _vp, _vp, _vp]
    lib.gs_pose_grad_reduce.argtypes = [_vp, C.c_int, C.c_int, _vp, _vp, _vp]
    lib.gs_pose_adam_step.argtypes = [_vp, _vp, _vp, C.c_int, C.POINTER(gs_adam), _vp, _vp]
    for name in ("gs_project", "gs_project_bf16", "gs_render_fwd_bwd_pose", "gs_spatial_order", "gs_pack_bf16", "gs_bin_tiles", "gs_render_fwd", "gs_render_bwd", "gs_nu_accumulate",
                 "gs_nu_finalize", "gs_pose_grad_reduce", "gs_pose_adam_step"):
        getattr(lib, name).restype = C.c_int
    return lib


lib = _load()


def last_error() -> str:
    return lib.gs_last_error().decode()


def _check(st: int) -> None:
    if st != GS_OK:
        raise GsError(st, last_error())


# ----------------------------------------------------------------- marshalling
def _ptr(t: Optional[torch.Tensor], dtype=None, name="tensor", numel=None):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{name} holds {t.numel()} elements, needs {numel}")
    return t.data_ptr()


def _stream(stream) -> Optional[int]:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def cameras(cams: Sequence) -> C.Array:
    arr = (gs_camera * len(cams))()
    for i, c in enumerate(cams):
        arr[i] = gs_camera(int(c.width), int(c.height), float(c.fx), float(c.fy), float(c.cx), float(c.cy),
                           float(getattr(c, "znear", 0.2)))
    return arr


@dataclass
class Gaussians:
    """Gaussian parameters as FP32 CUDA tensors ([N,3], [N,3], [N,4], [N], [N,3], [N])."""
    means: torch.Tensor
    log_scales: torch.Tensor
    quats: torch.Tensor
    opacity_logit: torch.Tensor
    colors: torch.Tensor
    nu: torch.Tensor

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def struct(self) -> gs_gaussians:
        n = self.n
        return gs_gaussians(n, _ptr(self.means, torch.float32, "means", 3 * n),
                            _ptr(self.log_scales, torch.float32, "log_scales", 3 * n),
                            _ptr(self.quats, torch.float32, "quats", 4 * n),
                            _ptr(self.opacity_logit, torch.float32, "opacity_logit", n),
                            _ptr(self.colors, torch.float32, "colors", 3 * n),
                            _ptr(self.nu, torch.float32, "nu", n))


def gs_project(g: Gaussians, cams, T_cw: torch.Tensor, opts: gs_opts, rec: torch.Tensor,
               tiles_touched: torch.Tensor, pose_jac: Optional[torch.Tensor], status: torch.Tensor,
               stream=None) -> None:
    F = len(cams)
    M = F * g.n
    proj = gs_projected(g.n, F, _ptr(rec, torch.float32, "rec", M * GS_REC_FLOATS),
                        _ptr(tiles_touched, torch.int32, "tiles_touched", M),
                        _ptr(pose_jac, torch.float32, "pose_jac", M * GS_JAC_FLOATS))
    _check(lib.gs_project(C.byref(g.struct()), F, cameras(cams), _ptr(T_cw, torch.float32, "T_cw", 12 * F),
                          C.byref(opts), C.byref(proj), _ptr(status, torch.int32, "status", 4), _stream(stream)))


@dataclass
class PackedGaussians:
    """16-bit storage (gs_gaussians_bf16): FP32 chunk boxes [ceil(N/256), 8] (lo
    xyz, step xyz, 0, 0), packed records [N, 16] (int16 tensor holding the bits:
    uint16 fixed-point mean, BF16 attributes) and the permutation (int32 [N])
    from packed order to the FP32 source order, or None."""
    anchors: torch.Tensor
    packed: torch.Tensor
    perm: Optional[torch.Tensor] = None

    @property
    def n(self) -> int:
        return int(self.packed.shape[0])

    def struct(self) -> gs_gaussians_bf16:
        n = self.n
        return gs_gaussians_bf16(n, _ptr(self.anchors, torch.float32, "anchors",
                                         8 * ((n + GS_BF16_CHUNK - 1) // GS_BF16_CHUNK)),
                                 _ptr(self.packed, torch.int16, "packed", 16 * n))


def gs_project_bf16(g: PackedGaussians, cams, T_cw: torch.Tensor, opts: gs_opts, rec: torch.Tensor,
                    tiles_touched: torch.Tensor, pose_jac: Optional[torch.Tensor], status: torch.Tensor,
                    stream=None) -> None:
    F = len(cams)
    M = F * g.n
    proj = gs_projected(g.n, F, _ptr(rec, torch.float32, "rec", M * GS_REC_FLOATS),
                        _ptr(tiles_touched, torch.int32, "tiles_touched", M),
                        _ptr(pose_jac, torch.float32, "pose_jac", M * GS_JAC_FLOATS))
    _check(lib.gs_project_bf16(C.byref(g.struct()), F, cameras(cams), _ptr(T_cw, torch.float32, "T_cw", 12 * F),
                               C.byref(opts), C.byref(proj), _ptr(status, torch.int32, "status", 4),
                               _stream(stream)))


def gs_spatial_order_workspace_size(n: int) -> int:
    return int(lib.gs_spatial_order_workspace_size(n))


def gs_spatial_order(means: torch.Tensor, perm: torch.Tensor, ws: torch.Tensor, status: torch.Tensor,
                     stream=None) -> None:
    n = means.shape[0]
    _check(lib.gs_spatial_order(_ptr(means, torch.float32, "means", 3 * n), n, _ptr(perm, torch.int32, "perm", n),
                                _ptr(ws, torch.uint8, "ws"), ws.numel(), _ptr(status, torch.int32, "status", 4),
                                _stream(stream)))


def gs_pack_bf16(src: Gaussians, perm: Optional[torch.Tensor], anchors: torch.Tensor, packed: torch.Tensor,
                 status: torch.Tensor, stream=None) -> None:
    n = src.n
    _check(lib.gs_pack_bf16(C.byref(src.struct()), _ptr(perm, torch.int32, "perm", n),
                            _ptr(anchors, torch.float32, "anchors", 8 * ((n + GS_BF16_CHUNK - 1) // GS_BF16_CHUNK)),
                            _ptr(packed, torch.int16, "packed", 16 * n), _ptr(status, torch.int32, "status", 4),
                            _stream(stream)))


def pack_bf16(src: Gaussians, spatial: bool = True) -> PackedGaussians:
    """Spatially orders (optional) and packs FP32 Gaussians into 16-bit storage."""
    n, dev = src.n, src.means.device
    status = torch.zeros(4, dtype=torch.int32, device=dev)
    perm = None
    if spatial:
        perm = torch.empty(n, dtype=torch.int32, device=dev)
        ws = torch.empty(max(1, gs_spatial_order_workspace_size(n)), dtype=torch.uint8, device=dev)
        gs_spatial_order(src.means, perm, ws, status)
    anchors = torch.empty((n + GS_BF16_CHUNK - 1) // GS_BF16_CHUNK, 8, dtype=torch.float32, device=dev)
    packed = torch.empty(n, 16, dtype=torch.int16, device=dev)
    gs_pack_bf16(src, perm, anchors, packed, status)
    return PackedGaussians(anchors, packed, perm)


def gs_bin_tiles_workspace_size(n_records: int, capacity: int) -> int:
    return int(lib.gs_bin_tiles_workspace_size(n_records, capacity))


def gs_bin_tiles(n_gaussians: int, cams, opts: gs_opts, rec: torch.Tensor, tiles_touched: torch.Tensor,
                 values: torch.Tensor, keys: Optional[torch.Tensor], ranges: torch.Tensor, status: torch.Tensor,
                 ws: torch.Tensor, stream=None, order: Optional[torch.Tensor] = None) -> None:
    F = len(cams)
    proj = gs_projected(n_gaussians, F, _ptr(rec, torch.float32, "rec"), _ptr(tiles_touched, torch.int32), None)
    cap = values.numel()
    if keys is not None and keys.numel() < cap:
        raise ValueError("keys must hold as many entries as values")
    tiles = gs_tiles(cap, ranges.numel() // 2, _ptr(values, torch.int32, "values"),
                     _ptr(keys, torch.int64, "keys"), _ptr(ranges, torch.int32, "ranges"),
                     _ptr(order, torch.int32, "order", ranges.numel() // 2))
    _check(lib.gs_bin_tiles(C.byref(proj), F, cameras(cams), C.byref(opts), C.byref(tiles),
                            _ptr(status, torch.int32, "status", 4), _ptr(ws, torch.uint8, "ws"), ws.numel(),
                            _stream(stream)))


def gs_project_bin(g, cams, T_cw: torch.Tensor, opts: gs_opts, rec: torch.Tensor, tiles_touched: torch.Tensor,
                   pose_jac: Optional[torch.Tensor], values: torch.Tensor, keys: Optional[torch.Tensor],
                   ranges: torch.Tensor, status: torch.Tensor, ws: torch.Tensor, stream=None,
                   order: Optional[torch.Tensor] = None) -> None:
    """gs_project (g: Gaussians) or gs_project_bf16 (g: PackedGaussians) and
    gs_bin_tiles in one call, the projection counting the pairs."""
    F = len(cams)
    M = F * g.n
    proj = gs_projected(g.n, F, _ptr(rec, torch.float32, "rec", M * GS_REC_FLOATS),
                        _ptr(tiles_touched, torch.int32, "tiles_touched", M),
                        _ptr(pose_jac, torch.float32, "pose_jac", M * GS_JAC_FLOATS))
    cap = values.numel()
    if keys is not None and keys.numel() < cap:
        raise ValueError("keys must hold as many entries as values")
    tiles = gs_tiles(cap, ranges.numel() // 2, _ptr(values, torch.int32, "values"),
                     _ptr(keys, torch.int64, "keys"), _ptr(ranges, torch.int32, "ranges"),
                     _ptr(order, torch.int32, "order", ranges.numel() // 2))
    fn = lib.gs_project_bin_bf16 if isinstance(g, PackedGaussians) else lib.gs_project_bin
    _check(fn(C.byref(g.struct()), F, cameras(cams), _ptr(T_cw, torch.float32, "T_cw", 12 * F), C.byref(opts),
              C.byref(proj), C.byref(tiles), _ptr(status, torch.int32, "status", 4), _ptr(ws, torch.uint8, "ws"),
              ws.numel(), _stream(stream)))


def gs_bin_tiles_noalloc(n_gaussians: int, cams, opts: gs_opts, rec: torch.Tensor, tiles_touched: torch.Tensor,
                         values: torch.Tensor, keys: Optional[torch.Tensor], ranges: torch.Tensor,
                         status: torch.Tensor, stream=None, order: Optional[torch.Tensor] = None) -> None:
    """gs_bin_tiles without a caller workspace (static device scratch; see gs.h)."""
    F = len(cams)
    proj = gs_projected(n_gaussians, F, _ptr(rec, torch.float32, "rec"), _ptr(tiles_touched, torch.int32), None)
    cap = values.numel()
    if keys is not None and keys.numel() < cap:
        raise ValueError("keys must hold as many entries as values")
    tiles = gs_tiles(cap, ranges.numel() // 2, _ptr(values, torch.int32, "values"),
                     _ptr(keys, torch.int64, "keys"), _ptr(ranges, torch.int32, "ranges"),
                     _ptr(order, torch.int32, "order", ranges.numel() // 2))
    _check(lib.gs_bin_tiles_noalloc(C.byref(proj), F, cameras(cams), C.byref(opts), C.byref(tiles),
                                    _ptr(status, torch.int32, "status", 4), _stream(stream)))


def _image(img: dict) -> gs_image:
    ints = ("n_last", "n_contrib", "median_pos", "dom_pos")
    return gs_image(*(_ptr(img.get(k), torch.int32 if k in ints else torch.float32, k)
                      for k in ("color", "depth", "alpha", "unc", "nu_map", "median", "T_final", "n_last",
                                "n_contrib", "median_pos", "dom_pos", "dom_weight")))


def gs_render_fwd(n_gaussians: int, cams, opts: gs_opts, rec: torch.Tensor, values: torch.Tensor,
                  ranges: torch.Tensor, obs_depth: Optional[torch.Tensor], out: dict, status: torch.Tensor,
                  stream=None, order: Optional[torch.Tensor] = None, queue: Optional[torch.Tensor] = None) -> None:
    F = len(cams)
    proj = gs_projected(n_gaussians, F, _ptr(rec, torch.float32, "rec"), None, None)  # touched not read
    tiles = gs_tiles(values.numel(), ranges.numel() // 2, _ptr(values, torch.int32), None,
                     _ptr(ranges, torch.int32), _ptr(order, torch.int32, "order", ranges.numel() // 2),
                     _ptr(queue, torch.int32, "queue", 2))
    _check(lib.gs_render_fwd(C.byref(proj), C.byref(tiles), F, cameras(cams),
                             _ptr(obs_depth, torch.float32, "obs_depth"), C.byref(opts), C.byref(_image(out)),
                             _ptr(status, torch.int32, "status", 4), _stream(stream)))


def gs_pose_partials_per_frame(mode: int, n_gaussians: int, cams, tile: int) -> int:
    return int(lib.gs_pose_partials_per_frame(mode, n_gaussians, len(cams), cameras(cams), tile))


def gs_render_bwd_workspace_size(n_records: int, mode: int) -> int:
    return int(lib.gs_render_bwd_workspace_size(n_records, mode))


def gs_render_bwd(n_gaussians: int, cams, opts: gs_opts, rec: torch.Tensor, pose_jac: Optional[torch.Tensor],
                  values: torch.Tensor, ranges: torch.Tensor, T_cw: Optional[torch.Tensor], g: Optional[Gaussians],
                  obs_depth: Optional[torch.Tensor], fwd: dict, dL: Optional[dict], loss: Optional[dict],
                  grads: Optional[dict], pose_partials: torch.Tensor, pose_grad: Optional[torch.Tensor],
                  status: torch.Tensor, ws: torch.Tensor, stream=None, order: Optional[torch.Tensor] = None,
                  queue: Optional[torch.Tensor] = None, touched: Optional[torch.Tensor] = None) -> None:
    """touched: the projection's tiles_touched, required in FULL mode (each
    record's visibility); POSE mode does not read it."""
    F = len(cams)
    if touched is None and opts.mode == GS_MODE_FULL:
        raise ValueError("gs_render_bwd: FULL mode needs the projection's tiles_touched (touched=)")
    tt = _ptr(touched, torch.int32, "touched", n_gaussians * F)  # POSE mode: may be None (not read)
    proj = gs_projected(n_gaussians, F, _ptr(rec, torch.float32, "rec"), tt,
                        _ptr(pose_jac, torch.float32, "pose_jac"))
    tiles = gs_tiles(values.numel(), ranges.numel() // 2, _ptr(values, torch.int32), None,
                     _ptr(ranges, torch.int32), _ptr(order, torch.int32, "order", ranges.numel() // 2),
                     _ptr(queue, torch.int32, "queue", 2))
    gl = None
    if loss is not None:
        gl = gs_loss(float(loss.get("w_color", 0.0)), float(loss.get("w_depth", 0.0)), float(loss.get("w_unc", 0.0)),
                     float(loss.get("w_nu", 0.0)), float(loss.get("unc_tau", 0.0)),
                     _ptr(loss.get("target_color"), torch.float32, "target_color"),
                     _ptr(loss.get("target_depth"), torch.float32, "target_depth"),
                     float(loss.get("w_align", 0.0)))
    gd = None
    if dL is not None:
        gd = gs_image_grad(*(_ptr(dL.get(k), torch.float32, "dL." + k)
                             for k in ("color", "depth", "alpha", "unc", "nu_map", "median")))
    gg = None
    if grads is not None:
        gg = gs_grads(*(_ptr(grads.get(k), torch.float32, "grads." + k)
                        for k in ("means", "log_scales", "quats", "opacity_logit", "colors", "nu")))
    _check(lib.gs_render_bwd(C.byref(proj), C.byref(tiles), F, cameras(cams), _ptr(T_cw, torch.float32, "T_cw"),
                             C.byref(g.struct()) if g is not None else None,
                             _ptr(obs_depth, torch.float32, "obs_depth"), C.byref(_image(fwd)),
                             C.byref(gd) if gd is not None else None, C.byref(gl) if gl is not None else None,
                             C.byref(opts), C.byref(gg) if gg is not None else None,
                             _ptr(pose_partials, torch.float32, "pose_partials"),
                             _ptr(pose_grad, torch.float64, "pose_grad", 6 * F),
                             _ptr(status, torch.int32, "status", 4), _ptr(ws, torch.uint8, "ws"), ws.numel(),
                             _stream(stream)))


def gs_nu_accumulate(n_gaussians: int, cams, rec: torch.Tensor, values: torch.Tensor, obs_depth: torch.Tensor,
                     fwd: dict, nu_num: torch.Tensor, nu_cnt: torch.Tensor, dominant: Optional[torch.Tensor],
                     status: torch.Tensor, stream=None) -> None:
    F = len(cams)
    proj = gs_projected(n_gaussians, F, _ptr(rec, torch.float32, "rec"), None, None)  # touched not read
    tiles = gs_tiles(values.numel(), 0, _ptr(values, torch.int32, "values"), None, None)
    _check(lib.gs_nu_accumulate(C.byref(proj), C.byref(tiles), F, cameras(cams),
                                _ptr(obs_depth, torch.float32, "obs_depth"), C.byref(_image(fwd)),
                                _ptr(nu_num, torch.float64, "nu_num", n_gaussians),
                                _ptr(nu_cnt, torch.int32, "nu_cnt", n_gaussians),
                                _ptr(dominant, torch.int32, "dominant"), _ptr(status, torch.int32, "status", 4),
                                _stream(stream)))


def gs_nu_finalize(nu_num: torch.Tensor, nu_cnt: torch.Tensor, nu: torch.Tensor, tau: float,
                   low_opacity_logit: float, opacity_logit: Optional[torch.Tensor], n_over: Optional[torch.Tensor],
                   status: torch.Tensor, stream=None) -> None:
    n = nu.numel()
    _check(lib.gs_nu_finalize(n, _ptr(nu_num, torch.float64, "nu_num", n), _ptr(nu_cnt, torch.int32, "nu_cnt", n),
                              _ptr(nu, torch.float32, "nu"), float(tau), float(low_opacity_logit),
                              _ptr(opacity_logit, torch.float32, "opacity_logit", n),
                              _ptr(n_over, torch.int32, "n_over", 1), _ptr(status, torch.int32, "status", 4),
                              _stream(stream)))


def _loss(loss: dict) -> gs_loss:
    return gs_loss(float(loss.get("w_color", 0.0)), float(loss.get("w_depth", 0.0)), float(loss.get("w_unc", 0.0)),
                   float(loss.get("w_nu", 0.0)), float(loss.get("unc_tau", 0.0)),
                   _ptr(loss.get("target_color"), torch.float32, "target_color"),
                   _ptr(loss.get("target_depth"), torch.float32, "target_depth"),
                   float(loss.get("w_align", 0.0)))


def gs_render_fwd_bwd_pose(n_gaussians: int, cams, opts: gs_opts, rec: torch.Tensor, pose_jac: torch.Tensor,
                           values: torch.Tensor, ranges: torch.Tensor, loss: dict, out: Optional[dict],
                           pose_partials: torch.Tensor, pose_grad: Optional[torch.Tensor], status: torch.Tensor,
                           ws: torch.Tensor, stream=None, order: Optional[torch.Tensor] = None,
                           adam_state: Optional[torch.Tensor] = None, adam: Optional[gs_adam] = None,
                           T_cw: Optional[torch.Tensor] = None) -> None:
    """Tracking pass: forward + POSE backward of the colour/depth loss in one launch,
    optionally followed (in the same launch) by the Adam step on the pose."""
    F = len(cams)
    proj = gs_projected(n_gaussians, F, _ptr(rec, torch.float32, "rec"), None,
                        _ptr(pose_jac, torch.float32, "pose_jac"))
    tiles = gs_tiles(values.numel(), ranges.numel() // 2, _ptr(values, torch.int32), None,
                     _ptr(ranges, torch.int32), _ptr(order, torch.int32, "order", ranges.numel() // 2))
    gl = _loss(loss)
    img = _image(out) if out is not None else None
    _check(lib.gs_render_fwd_bwd_pose(C.byref(proj), C.byref(tiles), F, cameras(cams), C.byref(gl), C.byref(opts),
                                      C.byref(img) if img is not None else None,
                                      _ptr(pose_partials, torch.float32, "pose_partials"),
                                      _ptr(pose_grad, torch.float64, "pose_grad", 6 * F),
                                      _ptr(adam_state, torch.float64, "adam_state", GS_POSE_STATE_DOUBLES * F),
                                      C.byref(adam) if adam is not None else None,
                                      _ptr(T_cw, torch.float32, "T_cw", 12 * F),
                                      _ptr(status, torch.int32, "status", 4), _ptr(ws, torch.uint8, "ws"), ws.numel(),
                                      _stream(stream)))


def gs_pose_grad_reduce(partials: torch.Tensor, n_frames: int, per_frame: int, pose_grad: torch.Tensor,
                        status: torch.Tensor, stream=None) -> None:
    _check(lib.gs_pose_grad_reduce(_ptr(partials, torch.float32, "partials", n_frames * per_frame * 12), n_frames,
                                   per_frame, _ptr(pose_grad, torch.float64, "pose_grad", 6 * n_frames),
                                   _ptr(status, torch.int32, "status", 4), _stream(stream)))


def gs_pose_adam_step(state: torch.Tensor, pose_grad: torch.Tensor, T_cw: torch.Tensor, n_frames: int,
                      adam: gs_adam, status: torch.Tensor, stream=None) -> None:
    _check(lib.gs_pose_adam_step(_ptr(state, torch.float64, "state", GS_POSE_STATE_DOUBLES * n_frames),
                                 _ptr(pose_grad, torch.float64, "pose_grad", 6 * n_frames),
                                 _ptr(T_cw, torch.float32, "T_cw", 12 * n_frames), n_frames, C.byref(adam),
                                 _ptr(status, torch.int32, "status", 4), _stream(stream)))
