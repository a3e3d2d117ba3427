"""FP64 CPU oracle of the CG-SLAM Gaussian rasterizer (arXiv 2403.16095).

TEST INFRASTRUCTURE ONLY: the product path never imports this package. Only the
test-suite, the smoke check and the benchmark's CPU-baseline leg use it.

The arithmetic lives in ``gs_oracle.c`` (plain C, FP64, OpenMP over image rows);
this module compiles it with gcc and marshals numpy arrays through ctypes.
Every function takes FP32 generator outputs and widens them to FP64 exactly.
"""

from __future__ import annotations

import ctypes as C
import dataclasses
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class _Scene(C.Structure):
    _fields_ = [("n", C.c_int), ("means", _dp), ("log_scales", _dp), ("quats", _dp),
                ("opacity_logit", _dp), ("colors", _dp), ("nu", _dp)]


class _Cam(C.Structure):
    _fields_ = [("width", C.c_int), ("height", C.c_int), ("fx", C.c_double), ("fy", C.c_double),
                ("cx", C.c_double), ("cy", C.c_double), ("znear", C.c_double)]


class _Opts(C.Structure):
    _fields_ = [("jclamp", C.c_double), ("nu_cull", C.c_double)]


class _Loss(C.Structure):
    _fields_ = [("w_color", C.c_double), ("w_depth", C.c_double), ("w_unc", C.c_double),
                ("w_nu", C.c_double), ("unc_tau", C.c_double), ("target_color", _dp),
                ("target_depth", _dp), ("w_align", C.c_double), ("mask", C.POINTER(C.c_ubyte))]


class _Image(C.Structure):
    _fields_ = [("color", _dp), ("depth", _dp), ("alpha", _dp), ("unc", _dp), ("nu_map", _dp),
                ("median", _dp), ("T_final", _dp), ("n_contrib", _ip), ("margins", _dp),
                ("dominant", _ip), ("dom_weight", _dp), ("dom_margin", _dp)]


class _Grads(C.Structure):
    _fields_ = [("means", _dp), ("log_scales", _dp), ("quats", _dp), ("opacity_logit", _dp),
                ("colors", _dp), ("nu", _dp), ("g_mean2d", _dp), ("g_conic", _dp),
                ("g_opacity", _dp), ("g_depth", _dp), ("pose", _dp)]


def build(force: bool = False) -> str:
    """Compile gs_oracle.c into _build/liboracle.so (gcc, -O2, OpenMP, IEEE math)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-fno-fast-math", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.orc_project.argtypes = [C.POINTER(_Scene), C.POINTER(_Cam), _dp, C.POINTER(_Opts),
                                     _dp, _dp, _dp, _dp, _ip, _ip, _ip]
        _lib.orc_render.argtypes = [C.POINTER(_Scene), C.POINTER(_Cam), _dp, C.POINTER(_Opts), _dp,
                                    C.c_int, C.POINTER(_Image)]
        _lib.orc_render_pixels.argtypes = [C.POINTER(_Scene), C.POINTER(_Cam), _dp, C.POINTER(_Opts),
                                           _dp, C.c_int, _ip, C.c_int, C.POINTER(_Image)]
        _lib.orc_fd_window.argtypes = [C.POINTER(_Scene), C.c_int, C.POINTER(_Cam), _dp, C.POINTER(_Opts),
                                       C.POINTER(_Loss), C.c_int, _ip, C.c_double, _dp, _ip]
        _lib.orc_loss_value.argtypes = [C.POINTER(_Scene), C.POINTER(_Cam), _dp, C.POINTER(_Opts),
                                        C.POINTER(_Loss), _dp, C.POINTER(C.c_uint64)]
        _lib.orc_grad.argtypes = [C.POINTER(_Scene), C.POINTER(_Cam), _dp, C.POINTER(_Opts),
                                  C.POINTER(_Loss), C.POINTER(_Grads), _dp]
        _lib.orc_bin_tiles.argtypes = [C.c_int, C.c_int, _ip, C.POINTER(C.c_float), C.c_int, C.c_int,
                                       _ip, _ip, _ip, C.c_longlong, C.POINTER(C.c_uint64),
                                       C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
        _lib.orc_bin_tiles.restype = C.c_longlong
        _lib.orc_adam_step.argtypes = [_dp, _dp, C.c_double, C.c_double, C.c_double, C.c_double,
                                       C.c_double]
        _lib.orc_set_threads.argtypes = [C.c_int]
        _lib.orc_get_threads.restype = C.c_int
    return _lib


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def threads() -> int:
    return int(lib().orc_get_threads())


# ----------------------------------------------------------------- helpers
def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _p(a, t=_dp):
    return None if a is None else a.ctypes.data_as(t)


class _Keep:
    """Holds FP64 copies alive while the C call runs."""

    def __init__(self, scene):
        self.arrs = [_f64(getattr(scene, k)) for k in
                     ("means", "log_scales", "quats", "opacity_logit", "colors", "nu")]
        self.s = _Scene(int(self.arrs[0].shape[0]), *(_p(a) for a in self.arrs))


def _cam(cam):
    return _Cam(int(cam.width), int(cam.height), float(cam.fx), float(cam.fy), float(cam.cx),
                float(cam.cy), float(cam.znear))


@dataclasses.dataclass
class LossSpec:
    """L = sum_p 1/(HW) [ m_p (w_color sum_ch |C-C*| + w_depth |D-D*|) + w_unc |U| + w_nu nu_map
                          + w_align |D_alpha - D_median| ],
    m_p = 1/(1 + nu_map/unc_tau) if unc_tau > 0 else 1 (held constant in the gradient)."""
    w_color: float = 1.0
    w_depth: float = 1.0
    w_unc: float = 0.0
    w_nu: float = 0.0
    unc_tau: float = 0.0
    target_color: np.ndarray | None = None   # [3,H,W]
    target_depth: np.ndarray | None = None   # [H,W] (also the sensor depth of U)
    w_align: float = 0.0                     # L_align of Eq. 12
    pixels: np.ndarray | None = None         # flat pixel indices y*W+x: only these enter the sum


class _KeepLoss:
    def __init__(self, L: LossSpec, n_pix: int | None = None):
        self.tc = None if L.target_color is None else _f64(L.target_color)
        self.td = None if L.target_depth is None else _f64(L.target_depth)
        self.mask = None
        if L.pixels is not None:
            assert n_pix is not None
            self.mask = np.zeros(n_pix, np.uint8)
            self.mask[np.asarray(L.pixels, np.int64)] = 1
        self.s = _Loss(L.w_color, L.w_depth, L.w_unc, L.w_nu, L.unc_tau, _p(self.tc), _p(self.td), L.w_align,
                       _p(self.mask, C.POINTER(C.c_ubyte)))


# ----------------------------------------------------------------- API
def project(scene, cam, T, jclamp=1.3, nu_cull=0.0):
    k = _Keep(scene)
    n = scene.n
    Tc = _f64(T).reshape(3, 4)
    out = dict(mean2d=np.zeros((n, 2)), conic=np.zeros((n, 3)), depth=np.zeros(n), opacity=np.zeros(n),
               radius=np.zeros(n, np.int32), rect=np.zeros((n, 4), np.int32), valid=np.zeros(n, np.int32))
    r = lib().orc_project(C.byref(k.s), C.byref(_cam(cam)), _p(Tc), C.byref(_Opts(jclamp, nu_cull)),
                          _p(out["mean2d"]), _p(out["conic"]), _p(out["depth"]), _p(out["opacity"]),
                          _p(out["radius"], _ip), _p(out["rect"], _ip), _p(out["valid"], _ip))
    assert r == 0
    out["valid"] = out["valid"].astype(bool)
    return out


def _image_bufs(n_pix, H=None, W=None):
    shp = (n_pix,) if H is None else (H, W)
    o = dict(color=np.zeros((3, *shp)), depth=np.zeros(shp), alpha=np.zeros(shp), unc=np.zeros(shp),
             nu_map=np.zeros(shp), median=np.zeros(shp), T_final=np.zeros(shp),
             n_contrib=np.zeros(shp, np.int32), margins=np.zeros((6, *shp)),
             dominant=np.zeros(shp, np.int32), dom_weight=np.zeros(shp), dom_margin=np.zeros(shp))
    im = _Image(*(_p(o[k], _ip if k in ("n_contrib", "dominant") else _dp) for k in
                  ("color", "depth", "alpha", "unc", "nu_map", "median", "T_final", "n_contrib", "margins",
                   "dominant", "dom_weight", "dom_margin")))
    return o, im


def render(scene, cam, T, obs_depth=None, mode="rect", jclamp=1.3, nu_cull=0.0):
    """Full image, FP64. mode 'rect' (rect-scatter lists) or 'brute' (scan every
    Gaussian per pixel). Returns planar arrays: color [3,H,W], others [H,W];
    margins [6,H,W] are the per-pixel decision margins (q vs 9, alpha vs 1/255,
    T' vs 1e-4, opacity*G vs 0.99, relative depth gap of neighbours, T' vs 0.5).
    dominant [H,W] is the Gaussian with the largest blend weight (-1: none),
    dom_weight that weight and dom_margin its relative lead over the runner-up."""
    k = _Keep(scene)
    Tc = _f64(T).reshape(3, 4)
    od = None if obs_depth is None else _f64(obs_depth)
    o, im = _image_bufs(None, cam.height, cam.width)
    r = lib().orc_render(C.byref(k.s), C.byref(_cam(cam)), _p(Tc), C.byref(_Opts(jclamp, nu_cull)),
                         _p(od), 1 if mode == "rect" else 0, C.byref(im))
    assert r == 0
    return o


def render_pixels(scene, cam, T, pix, obs_depth=None, jclamp=1.3, nu_cull=0.0, mode="brute"):
    """Sampled pixels (flat indices y*W+x): 'brute' scans every Gaussian for
    each pixel; 'rect' draws the candidates from the row lists, as render()
    does (cheaper when many pixels are sampled)."""
    k = _Keep(scene)
    Tc = _f64(T).reshape(3, 4)
    od = None if obs_depth is None else _f64(obs_depth)
    pix = np.ascontiguousarray(pix, dtype=np.int32)
    o, im = _image_bufs(len(pix))
    r = lib().orc_render_pixels(C.byref(k.s), C.byref(_cam(cam)), _p(Tc), C.byref(_Opts(jclamp, nu_cull)),
                                _p(od), len(pix), _p(pix, _ip), 1 if mode == "rect" else 0, C.byref(im))
    assert r == 0
    return o


def loss_value(scene, cam, T, L: LossSpec, jclamp=1.3, nu_cull=0.0):
    """(loss, decision hash) for one frame."""
    k = _Keep(scene)
    kl = _KeepLoss(L, cam.width * cam.height)
    Tc = _f64(T).reshape(3, 4)
    v = C.c_double(0)
    h = C.c_uint64(0)
    r = lib().orc_loss_value(C.byref(k.s), C.byref(_cam(cam)), _p(Tc), C.byref(_Opts(jclamp, nu_cull)),
                             C.byref(kl.s), C.byref(v), C.byref(h))
    assert r == 0
    return v.value, h.value


def grad(scene, cam, T, L: LossSpec, jclamp=1.3, nu_cull=0.0):
    """Loss, parameter gradients, per-Gaussian 2D gradients and the left se(3)
    pose gradient (rho, phi) for one frame, all FP64."""
    k = _Keep(scene)
    kl = _KeepLoss(L, cam.width * cam.height)
    n = scene.n
    Tc = _f64(T).reshape(3, 4)
    o = dict(means=np.zeros((n, 3)), log_scales=np.zeros((n, 3)), quats=np.zeros((n, 4)),
             opacity_logit=np.zeros(n), colors=np.zeros((n, 3)), nu=np.zeros(n),
             g_mean2d=np.zeros((n, 2)), g_conic=np.zeros((n, 3)), g_opacity=np.zeros(n),
             g_depth=np.zeros(n), pose=np.zeros(6))
    g = _Grads(*(_p(o[f]) for f in ("means", "log_scales", "quats", "opacity_logit", "colors", "nu",
                                     "g_mean2d", "g_conic", "g_opacity", "g_depth", "pose")))
    v = C.c_double(0)
    r = lib().orc_grad(C.byref(k.s), C.byref(_cam(cam)), _p(Tc), C.byref(_Opts(jclamp, nu_cull)),
                       C.byref(kl.s), C.byref(g), C.byref(v))
    assert r == 0
    o["loss"] = v.value
    return o


FD_PARAMS = (("means", 3), ("log_scales", 3), ("quats", 4), ("opacity_logit", 1), ("colors", 3), ("nu", 1))


def fd_window(scene, cams, Ts, losses, sel, h=1e-4, jclamp=1.3, nu_cull=0.0):
    """Central differences (h, FP64) of the window loss sum_f L_f over frames
    (cams[f], Ts[f], losses[f]) for all 15 parameters of each Gaussian in
    ``sel``, re-blending only the pixels the perturbed Gaussian can reach (the
    same value as differencing full-image loss_value() sums).

    Returns (fd [len(sel), 15], stable [len(sel), 15] bool) with the parameters
    in FD_PARAMS order; stable is False where some pixel's blend decisions or
    the sign of an absolute-value residual differ between the base and x +- h."""
    k = _Keep(scene)
    sel = np.ascontiguousarray(sel, dtype=np.int32)
    F = len(cams)
    camarr = (_Cam * F)(*[_cam(c) for c in cams])
    Tc = _f64(np.stack([np.asarray(T, np.float64).reshape(3, 4) for T in Ts]))
    keeps = [_KeepLoss(L, c.width * c.height) for L, c in zip(losses, cams)]
    larr = (_Loss * F)(*[kl.s for kl in keeps])
    fd = np.zeros((len(sel), 15))
    st = np.zeros((len(sel), 15), np.int32)
    r = lib().orc_fd_window(C.byref(k.s), F, camarr, _p(Tc), C.byref(_Opts(jclamp, nu_cull)), larr, len(sel),
                            _p(sel, _ip), float(h), _p(fd), _p(st, _ip))
    assert r == 0
    return fd, st.astype(bool)


def nu_estimate(scene, cams, Ts, obs_depths, tau=0.0, low_opacity=0.01, jclamp=1.3, nu_cull=0.0):
    """Per-Gaussian depth uncertainty of Eq. 13 over a keyframe window (Sec. 3.2).

    In frame f, pixel p is a dominated pixel of the Gaussian i with the largest
    blend weight w = alpha T on p (the first in blend order on ties); i receives
    w (D_p - d_i)^2 with D_p the sensor depth and d_i its camera-space depth in
    f. nu_i = (sum over the window) / (M_1 + ... + M_k), its dominated-pixel
    count; a Gaussian with no dominated pixel keeps its nu. With tau > 0, every
    Gaussian with nu_i > tau has its opacity lowered to ``low_opacity`` (its
    logit becomes min(logit, logit(low_opacity))).

    Returns num [N], cnt [N] (int64), nu [N], over [N] (bool), opacity_logit
    [N] and the per-frame oracle images (with their dominant maps)."""
    n = scene.n
    num = np.zeros(n)
    cnt = np.zeros(n, np.int64)
    images = []
    for cam, T, D in zip(cams, Ts, obs_depths):
        im = render(scene, cam, T, jclamp=jclamp, nu_cull=nu_cull)
        d = project(scene, cam, T, jclamp=jclamp, nu_cull=nu_cull)["depth"]
        dom = im["dominant"].reshape(-1)
        w = im["dom_weight"].reshape(-1)
        Dp = _f64(D).reshape(-1)
        sel = dom >= 0
        i = dom[sel]
        np.add.at(num, i, w[sel] * (Dp[sel] - d[i]) ** 2)
        np.add.at(cnt, i, 1)
        images.append(im)
    nu = _f64(scene.nu).copy()
    has = cnt > 0
    nu[has] = num[has] / cnt[has]
    over = nu > tau if tau > 0 else np.zeros(n, bool)
    logit = _f64(scene.opacity_logit).copy()
    low = np.log(low_opacity / (1.0 - low_opacity))
    logit[over] = np.minimum(logit[over], low)
    return dict(num=num, cnt=cnt, nu=nu, over=over, opacity_logit=logit, images=images)


# ------------------------------------------------------- BF16 storage
BF16_CHUNK = 256


def bf16_bits(x):
    """Round FP32 values to BF16 (nearest, ties to even), as uint16 bit patterns:
    the upper 16 bits of the FP32 pattern after adding half an ulp of BF16
    (0x7fff) plus the lowest kept bit, so that a tie rounds to the even neighbour."""
    u = np.ascontiguousarray(np.asarray(x, np.float32)).view(np.uint32).astype(np.uint64)
    keep = (u >> 16) & 1
    return ((u + 0x7FFF + keep) >> 16).astype(np.uint16)


def bf16_value(bits):
    """BF16 bit patterns -> FP32 (exact: the bits become the upper half)."""
    return (np.asarray(bits, np.uint32) << 16).view(np.float32)


def _spread3(v):
    out = np.zeros_like(v, dtype=np.uint64)
    for b in range(10):
        out |= ((v >> b) & 1) << (3 * b)
    return out


def spatial_order(means):
    """Permutation of the Gaussians in 30-bit Morton order of their FP32 means:
    per axis q = min(1023, floor((m - lo) * (1024 / (hi - lo)))) in FP32 (0 on a
    flat axis), code bits x, y, z interleaved from the lowest up; stable (ties by
    index)."""
    m = np.asarray(means, np.float32).reshape(-1, 3)
    if m.shape[0] == 0:
        return np.zeros(0, np.int64)
    lo, hi = m.min(axis=0), m.max(axis=0)
    code = np.zeros(m.shape[0], np.uint64)
    for k in range(3):
        ext = np.float32(hi[k] - lo[k])
        if ext > 0:
            sc = np.float32(np.float32(1024.0) / ext)
            q = np.float32(m[:, k] - lo[k]) * sc
            q = np.minimum(np.floor(q), 1023).astype(np.uint64)
        else:
            q = np.zeros(m.shape[0], np.uint64)
        code |= _spread3(q) << k
    return np.argsort(code, kind="stable")


def pack_bf16(scene, perm=None):
    """16-bit storage of FP32 Gaussians in the order perm. Per chunk of 256, from
    the bounding box [lo, hi] of its means: step = (hi - lo) / 65535 and
    q = rint((m - lo) / step) clamped to [0, 65535] in FP32 (q = 0 where step = 0);
    the other values rounded to BF16. Returns anchors float32 [C, 8] = (lo xyz,
    step xyz, 0, 0) and packed uint16 [N, 16] = (q xyz, log-scale, quaternion,
    opacity logit, RGB, nu, 0)."""
    n = scene.n
    order = np.arange(n) if perm is None else np.asarray(perm)
    f32 = {k: np.asarray(getattr(scene, k), np.float32)[order] for k in
           ("means", "log_scales", "quats", "opacity_logit", "colors", "nu")}
    C = (n + BF16_CHUNK - 1) // BF16_CHUNK
    anchors = np.zeros((C, 8), np.float32)
    q = np.zeros((n, 3), np.uint16)
    for c in range(C):
        sl = slice(c * BF16_CHUNK, (c + 1) * BF16_CHUNK)
        m = f32["means"][sl]
        lo, hi = m.min(axis=0), m.max(axis=0)
        step = (hi - lo) / np.float32(65535.0)
        anchors[c, 0:3], anchors[c, 3:6] = lo, step
        with np.errstate(divide="ignore", invalid="ignore"):
            t = (m - lo) / step
        t = np.where(step > 0, np.rint(t), 0.0)
        q[sl] = np.clip(t, 0, 65535).astype(np.uint16)
    vals = np.concatenate([f32["log_scales"], f32["quats"], f32["opacity_logit"][:, None], f32["colors"],
                           f32["nu"][:, None], np.zeros((n, 1), np.float32)], axis=1)
    return anchors, np.concatenate([q, bf16_bits(vals)], axis=1)


def unpack_bf16(anchors, packed):
    """The FP32 Gaussians that 16-bit storage represents (mean = lo + step * q,
    FP32 product then FP32 sum), as a synth.Scene of FP64 arrays."""
    import synth
    packed = np.asarray(packed, np.uint16)
    n = packed.shape[0]
    box = np.asarray(anchors, np.float32)[np.arange(n) // BF16_CHUNK]
    means = box[:, 0:3] + box[:, 3:6] * packed[:, 0:3].astype(np.float32)
    v = bf16_value(packed[:, 3:])
    return synth.Scene(*(np.asarray(x, np.float64) for x in
                         (means, v[:, 0:3], v[:, 3:7], v[:, 7], v[:, 8:11], v[:, 11])))


def bin_tiles(rect, depth_f32, n_per_frame, tile, cams, capacity=None):
    """Brute-force tile lists: (keys u64 [P], values u32 [P], ranges u32 [n_tiles,2])."""
    rect = np.ascontiguousarray(rect, dtype=np.int32)
    depth = np.ascontiguousarray(depth_f32, dtype=np.float32)
    tx = np.array([(c.width + tile - 1) // tile for c in cams], np.int32)
    ty = np.array([(c.height + tile - 1) // tile for c in cams], np.int32)
    toff = np.concatenate([[0], np.cumsum(tx * ty)[:-1]]).astype(np.int32)
    n_tiles = int((tx * ty).sum())
    n = rect.shape[0]
    cap = capacity if capacity is not None else int(n) * n_tiles if n * n_tiles < 50_000_000 else 50_000_000
    while True:
        keys = np.zeros(max(cap, 1), np.uint64)
        vals = np.zeros(max(cap, 1), np.uint32)
        ranges = np.zeros((n_tiles, 2), np.uint32)
        P = lib().orc_bin_tiles(n, n_per_frame, _p(rect, _ip), depth.ctypes.data_as(C.POINTER(C.c_float)),
                                tile, len(cams), _p(tx, _ip), _p(ty, _ip), _p(toff, _ip), cap,
                                keys.ctypes.data_as(C.POINTER(C.c_uint64)),
                                vals.ctypes.data_as(C.POINTER(C.c_uint32)),
                                ranges.ctypes.data_as(C.POINTER(C.c_uint32)))
        if P == -1 and capacity is None:
            cap *= 4
            continue
        assert P >= 0, P
        return keys[:P], vals[:P], ranges


def adam_step(state, grad6, lr_rot=0.0015, lr_trans=0.00215, beta1=0.9, beta2=0.999, eps=1e-8):
    """In-place FP64 Adam step on the pose state [R(9), t(3), m(6), v(6), step]."""
    assert state.dtype == np.float64 and state.shape == (25,)
    g = _f64(grad6)
    lib().orc_adam_step(_p(state), _p(g), lr_rot, lr_trans, beta1, beta2, eps)
    return state
