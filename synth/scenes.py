"""Seeded scene, camera and pose generators.

Every generator takes an explicit seed and uses ``numpy.random.Generator(PCG64)``.
The shapes follow the indoor RGB-D workloads of CG-SLAM (Sec. 4: Replica, TUM,
ScanNet style rooms); no dataset content is used, only those shapes:

* ``tiny_scene``      -- 128x96, 2,000 Gaussians in a slab in front of the camera.
* ``room_scene``      -- Gaussians on the walls/floor/ceiling of a 6x5x3 m room plus
                         axis-aligned boxes, colored by a procedural value-noise
                         texture so photometric gradients carry information.
* ``two_room_scene``  -- 10x8x3 m, two rooms sharing a wall with a door opening.

Camera convention (shared with both the oracle and the CUDA path, stated here as
an input contract): world->camera pose ``T_cw = [R | t]`` (3x4, row-major),
camera axes x right, y down, z forward; pixel (i, j) covers [i, i+1) x [j, j+1).
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Camera:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    znear: float = 0.2


@dataclasses.dataclass
class Scene:
    means: np.ndarray          # [N,3] float32 world positions
    log_scales: np.ndarray     # [N,3] float32
    quats: np.ndarray          # [N,4] float32 (w, x, y, z)
    opacity_logit: np.ndarray  # [N]   float32
    colors: np.ndarray         # [N,3] float32 RGB (degree-0)
    nu: np.ndarray             # [N]   float32 per-Gaussian uncertainty property

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def as_dict(self):
        return dataclasses.asdict(self)

    def subset(self, idx):
        return Scene(*(getattr(self, f.name)[idx] for f in dataclasses.fields(self)))


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _unit_quats(rng, n):
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


# ---------------------------------------------------------------- tiny scene
def tiny_scene(n: int = 2000, seed: int = 1001, width: int = 128, height: int = 96,
               focal: float = 100.0, unit_quats: bool = True):
    """128x96 / 2k-Gaussian scene: means x,y in U[-1,1], z in U[1,5] at identity
    pose; log-scales N(-3, 0.5); opacity logits N(0,1); RGB U[0,1]; nu U[0,0.1].
    Returns (scene, camera, T_cw)."""
    rng = _rng(seed)
    means = np.stack([rng.uniform(-1, 1, n), rng.uniform(-1, 1, n), rng.uniform(1, 5, n)], 1)
    log_scales = rng.normal(-3.0, 0.5, size=(n, 3))
    quats = _unit_quats(rng, n) if unit_quats else rng.normal(size=(n, 4))
    opacity_logit = rng.normal(0.0, 1.0, size=n)
    colors = rng.uniform(0, 1, size=(n, 3))
    nu = rng.uniform(0, 0.1, size=n)
    sc = Scene(*(a.astype(np.float32) for a in (means, log_scales, quats, opacity_logit, colors, nu)))
    cam = Camera(width, height, focal, focal, width / 2.0, height / 2.0)
    T = np.zeros((3, 4), np.float32)
    T[:3, :3] = np.eye(3, dtype=np.float32)
    return sc, cam, T


def fd_scene(n: int = 40, seed: int = 1100, width: int = 64, height: int = 48,
             focal: float = 60.0, n_edge: int = 4):
    """Small overlapping scene for finite-difference checks: larger Gaussians
    (log-scale N(-2.3, 0.3)) at z in U[2,4], plus ``n_edge`` Gaussians placed just
    outside the horizontal field of view whose footprints still reach into the
    image (they exercise the clamp of x/z in the projection Jacobian).
    Quaternions are NOT normalised so the normalisation is exercised too."""
    rng = _rng(seed)
    z = rng.uniform(2.0, 4.0, n)
    half_x = 0.5 * width / focal
    half_y = 0.5 * height / focal
    x = rng.uniform(-0.8, 0.8, n) * half_x * z
    y = rng.uniform(-0.8, 0.8, n) * half_y * z
    ze = rng.uniform(2.0, 3.0, n_edge)
    xe = np.where(rng.uniform(size=n_edge) < 0.5, -1.0, 1.0) * 1.38 * half_x * ze
    ye = rng.uniform(-0.5, 0.5, n_edge) * half_y * ze
    means = np.concatenate([np.stack([x, y, z], 1), np.stack([xe, ye, ze], 1)])
    m = n + n_edge
    log_scales = np.concatenate([rng.normal(-2.3, 0.3, size=(n, 3)), rng.normal(-1.3, 0.1, size=(n_edge, 3))])
    quats = rng.normal(size=(m, 4)) * rng.uniform(0.5, 2.0, size=(m, 1))
    opacity_logit = rng.normal(0.5, 1.0, size=m)
    colors = rng.uniform(0, 1, size=(m, 3))
    nu = rng.uniform(0, 0.1, size=m)
    sc = Scene(*(a.astype(np.float64) for a in (means, log_scales, quats, opacity_logit, colors, nu)))
    cam = Camera(width, height, focal, focal, width / 2.0, height / 2.0)
    T = np.zeros((3, 4))
    T[:3, :3] = np.eye(3)
    return sc, cam, T


def random_targets(cam: Camera, seed: int, n_frames: int = 1, depth_range=(1.0, 5.0)):
    """Per-pixel targets: color U[0,1]^3 planar [F,3,H,W], depth U[lo,hi] [F,H,W]."""
    rng = _rng(seed)
    col = rng.uniform(0, 1, size=(n_frames, 3, cam.height, cam.width)).astype(np.float32)
    dep = rng.uniform(depth_range[0], depth_range[1],
                      size=(n_frames, cam.height, cam.width)).astype(np.float32)
    return col, dep


# ------------------------------------------------------------ value noise
class _ValueNoise:
    """Multi-octave trilinear value noise: a procedural RGB texture of position."""

    def __init__(self, rng, lo, hi, cells=(0.5, 0.12), weights=(0.6, 0.4)):
        self.lo = np.asarray(lo, np.float64)
        self.octaves = []
        for cell, w in zip(cells, weights):
            shape = np.ceil((np.asarray(hi) - self.lo) / cell).astype(int) + 2
            self.octaves.append((cell, w, rng.uniform(0, 1, size=(*shape, 3))))

    def __call__(self, p):
        out = np.zeros((p.shape[0], 3))
        for cell, w, lat in self.octaves:
            g = (p - self.lo) / cell
            i0 = np.clip(np.floor(g).astype(int), 0, np.asarray(lat.shape[:3]) - 2)
            f = np.clip(g - i0, 0.0, 1.0)
            acc = np.zeros_like(out)
            for dx in (0, 1):
                for dy in (0, 1):
                    for dz in (0, 1):
                        wt = ((f[:, 0] if dx else 1 - f[:, 0]) * (f[:, 1] if dy else 1 - f[:, 1])
                              * (f[:, 2] if dz else 1 - f[:, 2]))
                        acc += wt[:, None] * lat[i0[:, 0] + dx, i0[:, 1] + dy, i0[:, 2] + dz]
            out += w * acc
        return out


# ------------------------------------------------------------ room scenes
def _box_faces(lo, hi, inward: bool, skip_bottom: bool = False):
    """Axis-aligned faces of a box as (origin, u-edge, v-edge) parallelograms."""
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    d = hi - lo
    faces = []
    for axis in range(3):
        for side in (0, 1):
            if skip_bottom and axis == 2 and side == 0:
                continue
            o = lo.copy()
            o[axis] = hi[axis] if side else lo[axis]
            a1, a2 = [a for a in range(3) if a != axis]
            e1 = np.zeros(3)
            e1[a1] = d[a1]
            e2 = np.zeros(3)
            e2[a2] = d[a2]
            faces.append((o, e1, e2))
    return faces


def _sample_faces(rng, faces, n, openings=()):
    """Uniform samples over a set of parallelogram faces, allocated by area.
    ``openings`` are axis-aligned boxes (lo, hi) whose interior is left empty."""
    areas = np.array([np.linalg.norm(np.cross(e1, e2)) for _, e1, e2 in faces])
    counts = np.floor(n * areas / areas.sum()).astype(int)
    counts[: n - counts.sum()] += 1
    pts = []
    for (o, e1, e2), c in zip(faces, counts):
        need = c
        chunk = []
        while need > 0:
            uv = rng.uniform(0, 1, size=(int(need * 1.3) + 16, 2))
            p = o + uv[:, :1] * e1 + uv[:, 1:] * e2
            keep = np.ones(len(p), bool)
            for olo, ohi in openings:
                keep &= ~np.all((p > np.asarray(olo)) & (p < np.asarray(ohi)), axis=1)
            p = p[keep][:need]
            chunk.append(p)
            need -= len(p)
        pts.append(np.concatenate(chunk) if chunk else np.zeros((0, 3)))
    return np.concatenate(pts)


def _finish_scene(rng, pts, log_scale_mu, log_scale_sd, lo, hi):
    n = pts.shape[0]
    perm = rng.permutation(n)          # no spatial order in the index
    pts = pts[perm]
    tex = _ValueNoise(rng, lo, hi)
    log_scales = rng.normal(log_scale_mu, log_scale_sd, size=(n, 3))
    quats = _unit_quats(rng, n)
    opacity_logit = rng.normal(1.0, 1.0, size=n)
    colors = np.clip(tex(pts), 0.0, 1.0)
    nu = rng.uniform(0.0, 0.1, size=n)
    return Scene(*(a.astype(np.float32) for a in (pts, log_scales, quats, opacity_logit, colors, nu)))


def room_scene(n: int, seed: int = 1002, size=(6.0, 5.0, 3.0), n_boxes: int = 20,
               log_scale=(-4.0, 0.4)):
    """Gaussians on the walls, floor and ceiling of a box room plus ``n_boxes``
    random axis-aligned boxes (sides U[0.2,1.0] m) resting on the floor, allocated
    in proportion to surface area and uniform on each face. World z is up."""
    rng = _rng(seed)
    W, D, H = size
    faces = _box_faces((0, 0, 0), (W, D, H), inward=True)
    for _ in range(n_boxes):
        s = rng.uniform(0.2, 1.0, size=3)
        cx = rng.uniform(s[0] / 2 + 0.05, W - s[0] / 2 - 0.05)
        cy = rng.uniform(s[1] / 2 + 0.05, D - s[1] / 2 - 0.05)
        faces += _box_faces((cx - s[0] / 2, cy - s[1] / 2, 0.0),
                            (cx + s[0] / 2, cy + s[1] / 2, s[2]), inward=False, skip_bottom=True)
    pts = _sample_faces(rng, faces, n)
    return _finish_scene(rng, pts, log_scale[0], log_scale[1], (0, 0, 0), size)


def two_room_scene(n: int, seed: int = 1004, size=(10.0, 8.0, 3.0), n_boxes: int = 30):
    """Two rooms side by side (shared wall at x = size/2 with a 1 m x 2 m door)."""
    rng = _rng(seed)
    W, D, H = size
    faces = _box_faces((0, 0, 0), (W, D, H), inward=True)
    faces.append((np.array([W / 2, 0.0, 0.0]), np.array([0.0, D, 0.0]), np.array([0.0, 0.0, H])))
    door = ((W / 2 - 0.01, D / 2 - 0.5, 0.0), (W / 2 + 0.01, D / 2 + 0.5, 2.0))
    for _ in range(n_boxes):
        s = rng.uniform(0.2, 1.0, size=3)
        cx = rng.uniform(s[0] / 2 + 0.05, W - s[0] / 2 - 0.05)
        cy = rng.uniform(s[1] / 2 + 0.05, D - s[1] / 2 - 0.05)
        faces += _box_faces((cx - s[0] / 2, cy - s[1] / 2, 0.0),
                            (cx + s[0] / 2, cy + s[1] / 2, s[2]), inward=False, skip_bottom=True)
    pts = _sample_faces(rng, faces, n, openings=[door])
    return _finish_scene(rng, pts, -4.0, 0.4, (0, 0, 0), size)


# ------------------------------------------------------------ cameras & poses
def look_at(center, target, up=(0.0, 0.0, 1.0)):
    """World->camera [R|t] (3x4, float64) for a camera at ``center`` looking at
    ``target`` with x right, y down, z forward."""
    c = np.asarray(center, float)
    d = np.asarray(target, float) - c
    d /= np.linalg.norm(d)
    r = np.cross(d, np.asarray(up, float))
    r /= np.linalg.norm(r)
    dn = np.cross(d, r)
    R = np.stack([r, dn, d])
    T = np.zeros((3, 4))
    T[:, :3] = R
    T[:, 3] = -R @ c
    return T


def room_track_poses(n_frames: int = 10, seed: int = 1002, size=(6.0, 5.0, 3.0)):
    """Ground-truth poses on a smooth path inside the room: height 1.2-1.8 m,
    sweeping yaw; returned as [F,3,4] float64."""
    rng = _rng(seed + 7)
    W, D, _ = size
    c0 = np.array([W * rng.uniform(0.35, 0.65), D * rng.uniform(0.35, 0.65)])
    yaw0 = rng.uniform(0, 2 * math.pi)
    poses = []
    for k in range(n_frames):
        s = k / max(1, n_frames - 1)
        pos = np.array([c0[0] + 0.4 * math.sin(2 * math.pi * s),
                        c0[1] + 0.3 * math.sin(4 * math.pi * s),
                        1.5 + 0.3 * math.sin(2 * math.pi * s + 1.0)])
        yaw = yaw0 + 1.2 * s
        pitch = -0.15 + 0.1 * math.sin(3 * math.pi * s)
        fwd = np.array([math.cos(yaw) * math.cos(pitch), math.sin(yaw) * math.cos(pitch), math.sin(pitch)])
        poses.append(look_at(pos, pos + fwd))
    return np.stack(poses)


def circle_poses(n_frames: int = 8, seed: int = 1003, center=(3.0, 2.5, 1.5), diameter: float = 3.0):
    """Keyframes on a circle (seeded phase), each looking at the circle's center."""
    rng = _rng(seed + 11)
    phase = rng.uniform(0, 2 * math.pi)
    c = np.asarray(center, float)
    poses = []
    for k in range(n_frames):
        a = phase + 2 * math.pi * k / n_frames
        pos = c + np.array([0.5 * diameter * math.cos(a), 0.5 * diameter * math.sin(a), 0.0])
        poses.append(look_at(pos, c + np.array([0.0, 0.0, -0.2])))
    return np.stack(poses)


def mixed_resolution_cameras():
    """6x 320x240 (f=300), 6x 640x480 (f=600), 4x 1200x680 (f=1125), principal
    point at the image center."""
    cams = [Camera(320, 240, 300.0, 300.0, 160.0, 120.0) for _ in range(6)]
    cams += [Camera(640, 480, 600.0, 600.0, 320.0, 240.0) for _ in range(6)]
    cams += [Camera(1200, 680, 1125.0, 1125.0, 600.0, 340.0) for _ in range(4)]
    return cams


def _rodrigues(axis_angle):
    th = float(np.linalg.norm(axis_angle))
    if th == 0.0:
        return np.eye(3)
    k = np.asarray(axis_angle, float) / th
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + math.sin(th) * K + (1 - math.cos(th)) * (K @ K)


def jitter_pose(T, seed: int, trans: float = 0.02, rot_deg: float = 1.0):
    """Start pose = ground truth moved by ``trans`` metres in a random direction
    and rotated by ``rot_deg`` degrees about a random axis (camera frame)."""
    rng = _rng(seed)
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    a = rng.normal(size=3)
    a /= np.linalg.norm(a)
    dR = _rodrigues(a * math.radians(rot_deg))
    out = np.array(T, dtype=np.float64, copy=True)
    out[:, :3] = dR @ out[:, :3]
    out[:, 3] = dR @ out[:, 3] + trans * d
    return out


# ------------------------------------------------------------ named workloads
def workload(name: str):
    """The named synthetic workloads (each seeded with 1000 + its index)."""
    if name == "tiny":
        sc, cam, T = tiny_scene()
        return dict(scene=sc, cams=[cam], poses=T[None].astype(np.float64))
    if name == "track":
        sc = room_scene(300_000, seed=1002)
        cam = Camera(640, 480, 600.0, 600.0, 320.0, 240.0)
        return dict(scene=sc, cams=[cam], poses=room_track_poses(10, seed=1002))
    if name == "mapping":
        sc = room_scene(1_000_000, seed=1003)
        cam = Camera(640, 480, 600.0, 600.0, 320.0, 240.0)
        return dict(scene=sc, cams=[cam] * 8, poses=circle_poses(8, seed=1003))
    if name == "uneven":
        sc = two_room_scene(2_000_000, seed=1004)
        cams = mixed_resolution_cameras()
        rng = _rng(1004 + 5)
        poses = []
        for k in range(len(cams)):
            pos = np.array([rng.uniform(1.0, 9.0), rng.uniform(1.0, 7.0), rng.uniform(1.2, 1.8)])
            yaw = rng.uniform(0, 2 * math.pi)
            poses.append(look_at(pos, pos + np.array([math.cos(yaw), math.sin(yaw), -0.1])))
        return dict(scene=sc, cams=cams, poses=np.stack(poses))
    if name == "precision":
        sc = room_scene(5_000_000, seed=1005)
        cam = Camera(1200, 680, 600.0, 600.0, 600.0, 340.0)
        return dict(scene=sc, cams=[cam], poses=room_track_poses(100, seed=1005))
    raise KeyError(name)
