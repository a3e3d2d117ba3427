"""GPU parity of the projection (Eq. 1-2) and the tile binning (Sec. 3.1
pre-sort) against the FP64 oracle, called through the C ABI."""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_util import f32_scene, poses_gpu, rec_fields, to_gpu_gaussians

pytestmark = pytest.mark.gpu


def _rast(cams, n, tile=16, mode=None, capacity=None, keep_keys=True):
    from paper_2403_16095_b300 import Rasterizer
    from paper_2403_16095_b300 import _abi as A
    return Rasterizer(cams, n, tile=tile, mode=A.GS_MODE_POSE if mode is None else mode, capacity=capacity,
                      keep_keys=keep_keys)


def _rect_margin(ora):
    """Distance of every floating rect bound to the integer it is rounded to."""
    con = ora["conic"]
    # largest eigenvalue of the 2D covariance = 1 / smallest eigenvalue of the conic
    tr, det = con[:, 0] + con[:, 2], con[:, 0] * con[:, 2] - con[:, 1] ** 2
    lam_min_conic = 0.5 * tr - np.sqrt(np.maximum(0.25 * tr ** 2 - det, 0))
    r3 = 3.0 * np.sqrt(1.0 / np.maximum(lam_min_conic, 1e-300))
    m = np.abs(r3 - np.round(r3))
    r = ora["radius"]
    for c in (0, 1):
        for s in (-1, 1):
            v = ora["mean2d"][:, c] - 0.5 + s * r
            m = np.minimum(m, np.abs(v - np.round(v)))
    return m


def test_projection_matches_oracle():
    sc, cam, T = synth.tiny_scene()
    g = to_gpu_gaussians(sc)
    r = _rast([cam], sc.n)
    r.reset_status()
    r.project(g, poses_gpu(T))
    torch.cuda.synchronize()
    got = rec_fields(r)
    ora = oracle.project(f32_scene(sc), cam, T)
    v = ora["valid"]
    assert np.array_equal(got["valid"], v)
    np.testing.assert_allclose(got["mean2d"][v], ora["mean2d"][v], rtol=1e-6, atol=2e-4)
    np.testing.assert_allclose(got["depth"][v], ora["depth"][v], rtol=1e-6)
    np.testing.assert_allclose(got["opacity"][v], ora["opacity"][v], rtol=1e-6, atol=1e-7)
    scale = np.abs(ora["conic"][v]).max(1, keepdims=True)
    np.testing.assert_allclose(got["conic"][v] / scale, ora["conic"][v] / scale, rtol=0, atol=2e-5)
    same = np.all(got["rect"][v] == ora["rect"][v], axis=1) & (got["radius"][v] == ora["radius"][v])
    bad = ~same
    assert bad.sum() <= 2
    assert np.all(_rect_margin(ora)[v][bad] < 1e-3), "rect mismatch away from a rounding boundary"


def _exp_pose(T, xi):
    rho, phi = xi[:3], xi[3:]
    th = np.linalg.norm(phi)
    K = np.array([[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]])
    R = np.eye(3) if th == 0 else np.eye(3) + math.sin(th) / th * K + (1 - math.cos(th)) / th ** 2 * K @ K
    out = np.zeros((3, 4))
    out[:, :3] = R @ T[:, :3]
    out[:, 3] = R @ T[:, 3] + rho
    return out


def test_pose_jacobian_matches_oracle_finite_differences():
    """The forward-mode d(mean2d, conic, z)/d(rho, phi) of gs_project (POSE mode)
    equals central differences of the FP64 oracle projection under Exp(xi) T."""
    sc, cam, _ = synth.fd_scene()
    T = _exp_pose(np.c_[np.eye(3), np.zeros(3)], np.array([0.03, -0.02, 0.1, 0.05, -0.03, 0.02]))
    g = to_gpu_gaussians(sc)
    r = _rast([cam], sc.n)
    r.reset_status()
    r.project(g, poses_gpu(T))
    torch.cuda.synchronize()
    jac = r.jac.view(-1, 6, 6).cpu().numpy().astype(np.float64)
    valid = rec_fields(r)["valid"]
    s64 = f32_scene(sc)
    h = 1e-6
    fd = np.zeros((sc.n, 6, 6))
    for k in range(6):
        xi = np.zeros(6)
        xi[k] = h
        p = oracle.project(s64, cam, _exp_pose(T, xi))
        m = oracle.project(s64, cam, _exp_pose(T, -xi))
        for arr, sl in (("mean2d", slice(0, 2)), ("conic", slice(2, 5))):
            fd[:, sl, k] = (p[arr] - m[arr]) / (2 * h)
        fd[:, 5, k] = (p["depth"] - m["depth"]) / (2 * h)
    for row in range(6):
        scale = np.abs(fd[valid, row, :]).max(axis=1, keepdims=True) + 1e-30
        err = np.abs(jac[valid, row, :] - fd[valid, row, :]) / scale
        assert err.max() < 2e-3, (row, err.max())


# ------------------------------------------------------------------ binning
def _synthetic_records(n, cams, tile, seed, ties=True):
    """Records with random pixel rects and depths: ties=True draws from four
    depths (runs of equal depth of hundreds of keys), "short" from n // 3
    depths (runs of a few keys), False from a continuous range."""
    rng = np.random.default_rng(seed)
    F = len(cams)
    rec = np.zeros((F * n, 16), np.float32)
    rect = np.zeros((F * n, 4), np.int32)
    for f, c in enumerate(cams):
        x0 = rng.integers(0, c.width, n)
        y0 = rng.integers(0, c.height, n)
        rect[f * n:(f + 1) * n] = np.c_[x0, y0, np.minimum(c.width - 1, x0 + rng.integers(0, 50, n)),
                                        np.minimum(c.height - 1, y0 + rng.integers(0, 50, n))]
    culled = rng.uniform(size=F * n) < 0.1
    rect[culled] = [1, 1, 0, 0]
    if ties == "short":
        depth = (0.5 + 0.001 * rng.integers(0, max(1, n // 3), F * n)).astype(np.float32)
    elif ties:
        depth = rng.choice(np.float32([0.25, 1.0, 1.5, 7.0]), F * n)
    else:
        depth = rng.uniform(0.2, 50.0, F * n).astype(np.float32)
    rec[:, 6] = depth
    rec.view(np.int32)[:, 12:16] = rect
    ok = rect[:, 0] <= rect[:, 2]
    touched = np.where(ok, (rect[:, 2] // tile - rect[:, 0] // tile + 1) * (rect[:, 3] // tile - rect[:, 1] // tile + 1), 0)
    return rec, rect, depth, touched.astype(np.int32)


@pytest.mark.parametrize("cams,tile,ties,n", [
    ([synth.Camera(128, 96, 1, 1, 0, 0)], 16, True, 3000),                  # 48 tiles
    ([synth.Camera(640, 480, 1, 1, 0, 0)], 16, False, 3000),                # 1200 tiles
    ([synth.Camera(640, 480, 1, 1, 0, 0)], 16, "short", 20000),             # 1200 tiles, counters a line apart
    # 6,450 tiles (a batch of more than 2,048: ballot peers in the shared-memory
    # passes) with lists of ~600 keys
    ([synth.Camera(1200, 680, 1, 1, 0, 0)] * 2, 16, "short", 300000),
    ([synth.Camera(1200, 680, 1, 1, 0, 0)], 8, True, 3000),                 # 12750 tiles
    ([synth.Camera(100, 70, 1, 1, 0, 0), synth.Camera(37, 53, 1, 1, 0, 0),
      synth.Camera(64, 64, 1, 1, 0, 0)], 16, True, 3000),                   # uneven frames, ragged
    # lists of more than 2048 keys (radix path over the depth digits):
    ([synth.Camera(16, 16, 1, 1, 0, 0)], 16, True, 3000),                   # one tile; long equal-depth runs
    ([synth.Camera(16, 16, 1, 1, 0, 0)], 16, "short", 9000),                # runs of a few equal depths
    ([synth.Camera(40, 24, 1, 1, 0, 0)], 16, False, 20000),                 # 6 tiles, ~10k keys each
    ([synth.Camera(48, 40, 1, 1, 0, 0), synth.Camera(16, 16, 1, 1, 0, 0)], 8, "short", 5000),
    # lists of 2,049-4,096 keys (radix passes in global memory)
    ([synth.Camera(16, 16, 1, 1, 0, 0)], 16, False, 3500),
    ([synth.Camera(16, 16, 1, 1, 0, 0)], 16, "short", 4000),
    # lists of 1,025-2,048 keys (radix sort in shared memory), with short runs of
    # equal depth and with long ones (full-sort fallback)
    ([synth.Camera(16, 16, 1, 1, 0, 0)], 16, "short", 1800),
    ([synth.Camera(16, 16, 1, 1, 0, 0)], 16, True, 1800),
    ([synth.Camera(16, 16, 1, 1, 0, 0)], 16, False, 1300),
])
def test_bin_tiles_bit_exact(cams, tile, ties, n):
    rec, rect, depth, touched = _synthetic_records(n, cams, tile, seed=len(cams) * 7 + tile, ties=ties)
    r = _rast(cams, n, tile=tile, capacity=int(touched.sum()) + 17)
    r.rec.copy_(torch.from_numpy(rec.reshape(-1)))
    r.touched.copy_(torch.from_numpy(touched))
    r.reset_status()
    r.bin()
    torch.cuda.synchronize()
    code, P = r.read_status()
    assert code == 0 and P == touched.sum()
    keys, vals, ranges = oracle.bin_tiles(rect, depth, n, tile, cams)
    assert np.array_equal(r.keys[:P].cpu().numpy().view(np.uint64), keys)
    assert np.array_equal(r.values[:P].cpu().numpy().view(np.uint32), vals)
    got = r.ranges.view(-1, 2).cpu().numpy().view(np.uint32)
    full = ranges[:, 1] > ranges[:, 0]
    assert np.array_equal(got[full], ranges[full])          # non-empty tiles: exact [start, end)
    assert np.all(got[~full, 0] == got[~full, 1])            # empty tiles: any start == end
    # launch order: every tile once, list lengths (bucketed by 4) non-increasing
    order = r.order.cpu().numpy()
    assert np.array_equal(np.sort(order), np.arange(len(ranges)))
    lens = (ranges[:, 1] - ranges[:, 0]).astype(np.int64)
    b = np.minimum(lens[order] >> 2, 1023)
    assert np.all(np.diff(b) <= 0)


def test_bin_tiles_capacity_overflow_sets_status():
    cams = [synth.Camera(128, 96, 1, 1, 0, 0)]
    n = 500
    rec, rect, depth, touched = _synthetic_records(n, cams, 16, seed=3)
    P = int(touched.sum())
    r = _rast(cams, n, capacity=P - 1)
    r.rec.copy_(torch.from_numpy(rec.reshape(-1)))
    r.touched.copy_(torch.from_numpy(touched))
    r.reset_status()
    r.bin()
    r.forward()  # must be a no-op after the overflow
    torch.cuda.synchronize()
    code, need = r.read_status()
    from paper_2403_16095_b300 import _abi as A
    assert code == A.GS_ERR_CAPACITY and need == P
    r.set_capacity(need)
    r.reset_status()
    r.bin()
    torch.cuda.synchronize()
    assert r.read_status() == (0, P)


def test_bin_tiles_all_culled():
    cams = [synth.Camera(64, 48, 1, 1, 0, 0)]
    n = 100
    rec = np.zeros((n, 16), np.float32)
    rec.view(np.int32)[:, 12:16] = [1, 1, 0, 0]
    r = _rast(cams, n, capacity=8)
    r.rec.copy_(torch.from_numpy(rec.reshape(-1)))
    r.touched.zero_()
    r.reset_status()
    r.bin()
    torch.cuda.synchronize()
    assert r.read_status() == (0, 0)
    assert int(r.ranges.abs().sum()) == 0


def test_end_to_end_tile_lists_match_oracle_projection():
    """GPU projection + GPU binning vs oracle binning of the FP64 projection:
    identical per-tile lists except for Gaussians whose rect sits within FP32
    rounding of a pixel boundary, or whose depths tie in FP32."""
    sc, cam, T = synth.tiny_scene()
    g = to_gpu_gaussians(sc)
    r = _rast([cam], sc.n, capacity=64)
    r.render(g, poses_gpu(T))  # grows the pair buffer after the first overflow
    torch.cuda.synchronize()
    assert r.read_status()[0] == 0
    ora = oracle.project(f32_scene(sc), cam, T)
    rect = np.where(ora["valid"][:, None], ora["rect"], np.array([1, 1, 0, 0]))
    keys, vals, ranges = oracle.bin_tiles(rect, ora["depth"].astype(np.float32), sc.n, 16, [cam])
    P = r.read_status()[1]
    gv = r.values[:P].cpu().numpy()
    gr = r.ranges.view(-1, 2).cpu().numpy()
    margin = _rect_margin(ora)
    for t in range(gr.shape[0]):
        a = gv[gr[t, 0]:gr[t, 1]]
        b = vals[ranges[t, 0]:ranges[t, 1]].astype(np.int64)
        if np.array_equal(a, b):
            continue
        diff = np.setxor1d(a, b)
        assert np.all(margin[diff] < 1e-3), (t, diff)
        common = [x for x in a if x in set(b)]
        assert common == [x for x in b if x in set(a)], t


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("pose_mode", [True, False])
def test_project_bin_equals_project_then_bin(storage, pose_mode):
    """gs_project_bin (the projection kernel counts the pairs and the binning
    skips its count pass) writes records, tile counts, pose Jacobians and tile
    lists bit-identical to gs_project followed by gs_bin_tiles, on three frames
    of uneven size, in FP32 and in 16-bit storage."""
    from paper_2403_16095_b300 import pack_bf16
    from paper_2403_16095_b300 import _abi as A
    sc = synth.room_scene(60_000, seed=1411)
    cams = [synth.Camera(320, 240, 300.0, 300.0, 160.0, 120.0), synth.Camera(160, 120, 150.0, 150.0, 80.0, 60.0),
            synth.Camera(200, 152, 190.0, 190.0, 100.0, 76.0)]
    T = np.stack(synth.room_track_poses(3, seed=1411))
    g = to_gpu_gaussians(sc)
    if storage == "bf16":
        g = pack_bf16(g)
    mode = A.GS_MODE_POSE if pose_mode else A.GS_MODE_FWD
    out = []
    for fused in (False, True):
        r = _rast(cams, sc.n, mode=mode, capacity=2_000_000)
        r.reset_status()
        if fused:
            r.project_bin(g, poses_gpu(T))
        else:
            r.project(g, poses_gpu(T))
            r.bin()
        torch.cuda.synchronize()
        code, P = r.read_status()
        assert code == 0 and P > 1000
        out.append((r, P))
    (ra, Pa), (rb, Pb) = out
    assert Pa == Pb
    fa, fb = rec_fields(ra), rec_fields(rb)
    assert np.array_equal(fa["rect"], fb["rect"])
    vis = fa["valid"]
    assert vis.sum() > 100
    assert np.array_equal(ra.rec.view(-1, 16).cpu().numpy()[vis].view(np.int32),
                          rb.rec.view(-1, 16).cpu().numpy()[vis].view(np.int32))
    assert torch.equal(ra.touched, rb.touched)
    if pose_mode:
        ja, jb = ra.jac.view(-1, 36).cpu().numpy()[vis], rb.jac.view(-1, 36).cpu().numpy()[vis]
        assert np.array_equal(ja.view(np.int32), jb.view(np.int32))
    assert torch.equal(ra.values[:Pa], rb.values[:Pb])
    assert torch.equal(ra.keys[:Pa], rb.keys[:Pb])
    assert torch.equal(ra.ranges, rb.ranges)
    # launch order: tiles within one length bucket come in the order the scan's
    # shared-memory atomics hand out (any order is valid); the buckets match
    lens = (rb.ranges.view(-1, 2)[:, 1] - rb.ranges.view(-1, 2)[:, 0]).cpu().numpy().astype(np.int64)
    for r in (ra, rb):
        order = r.order.cpu().numpy()
        assert np.array_equal(np.sort(order), np.arange(len(lens)))
        assert np.all(np.diff(np.minimum(lens[order] >> 2, 1023)) <= 0)
    assert np.array_equal(np.minimum(lens[ra.order.cpu().numpy()] >> 2, 1023),
                          np.minimum(lens[rb.order.cpu().numpy()] >> 2, 1023))


@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 64, 65, 128, 129, 255, 256, 257, 511, 512, 513])
def test_bin_tiles_list_length_boundaries(n):
    """One tile holding exactly n pairs, across the boundaries of the sort paths
    (one warp in registers with 1, 2, 4 or 8 keys per lane below 256; a CTA
    bitonic network from 256 to 512 keys; the shared-memory radix sort above),
    with ties: keys equal the oracle's."""
    cams = [synth.Camera(16, 16, 1, 1, 0, 0)]
    rng = np.random.default_rng(9000 + n)
    rec = np.zeros((n, 16), np.float32)
    rect = np.tile(np.int32([[2, 3, 9, 12]]), (n, 1))
    depth = (0.5 + 0.01 * rng.integers(0, max(1, n // 2), n)).astype(np.float32)
    rec[:, 6] = depth
    rec.view(np.int32)[:, 12:16] = rect
    touched = np.ones(n, np.int32)
    r = _rast(cams, n, tile=16, capacity=n + 5)
    r.rec.copy_(torch.from_numpy(rec.reshape(-1)))
    r.touched.copy_(torch.from_numpy(touched))
    r.reset_status()
    r.bin()
    torch.cuda.synchronize()
    code, P = r.read_status()
    assert code == 0 and P == n
    keys, vals, ranges = oracle.bin_tiles(rect, depth, n, 16, cams)
    assert np.array_equal(r.keys[:P].cpu().numpy().view(np.uint64), keys)
    assert np.array_equal(r.values[:P].cpu().numpy().view(np.uint32), vals)


@pytest.mark.parametrize("case", ["no_gaussians", "all_behind"])
def test_project_bin_empty_inputs(case):
    """gs_project_bin with no Gaussians, or with every Gaussian behind the camera:
    status OK, no pairs, every tile empty."""
    from paper_2403_16095_b300 import Gaussians
    from paper_2403_16095_b300 import _abi as A
    cam = synth.Camera(40, 30, 30, 30, 20, 15)
    T = np.c_[np.eye(3), np.zeros(3)]
    if case == "no_gaussians":
        e = torch.zeros(0, device="cuda")
        g = Gaussians(e.view(0, 3), e.view(0, 3), torch.zeros(0, 4, device="cuda"), e, e.view(0, 3), e)
        n = 0
    else:
        sc, _, _ = synth.tiny_scene(n=50, seed=1203)
        sc = synth.Scene(sc.means * np.float32([1, 1, -1]), sc.log_scales, sc.quats, sc.opacity_logit, sc.colors,
                         sc.nu)
        g, n = to_gpu_gaussians(sc), sc.n
    r = _rast([cam], n, mode=A.GS_MODE_POSE, capacity=64)
    r.reset_status()
    r.project_bin(g, poses_gpu(T))
    torch.cuda.synchronize()
    assert r.read_status() == (0, 0)
    rg = r.ranges.view(-1, 2).cpu().numpy()
    assert np.all(rg[:, 0] == rg[:, 1])
