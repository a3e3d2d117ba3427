"""Mapping-side uses of the backward (GPU vs FP64 oracle):

* f1 -- the median-depth output (Eq. 7-8) is differentiable and L_align
  (Eq. 12) flows through autograd to the median Gaussian's depth;
* f3 -- a sliding window of keyframes (Eq. 21, k = 4) rendered and
  differentiated in ONE launch: parameter gradients summed over the frames and
  one se(3) gradient per keyframe;
* the GPU gradient of the autograd path against central finite differences of
  the FP64 oracle loss (h = 1e-4 on the FP64 scene) on sampled Gaussians.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_util import PARAMS, f32_scene, poses_gpu, to_gpu_gaussians

pytestmark = pytest.mark.gpu


def _rel(name, got, want, elem=1e-4, norm=1e-5, n_flip=0):
    """Per-array check relative to the array's largest oracle magnitude. A pixel
    whose FP32 decision differs from FP64 (oracle decision margin < 1e-5, e.g. T
    crossing 0.5 for the median) hands its contribution to a different Gaussian:
    the 2 * n_flip rows with the largest error are exempt."""
    scale = np.abs(want).max()
    d = np.asarray(got, np.float64) - want
    rows = np.abs(d).reshape(d.shape[0], -1).max(1) if d.ndim else np.abs(d).reshape(1)
    keep = np.ones(rows.shape[0], bool)
    if n_flip:
        keep[np.argsort(-rows)[:2 * n_flip]] = False
    dk, wk = d[keep], np.asarray(want)[keep]
    e_max, e_norm = np.abs(dk).max() / scale, np.linalg.norm(dk) / np.linalg.norm(wk)
    print(f"{name}: max {e_max:.2e} norm {e_norm:.2e} (exempt rows {int((~keep).sum())})")
    assert e_max < elem and e_norm < norm, (name, e_max, e_norm)


def _n_flip(sc, cam, T, gpu_img):
    """Pixels where an FP32 decision differs from the FP64 one: some rendered
    channel (median included) differs from the oracle by more than 1e-4. Each
    must sit at an oracle decision margin below 1e-5."""
    ora = oracle.render(f32_scene(sc), cam, T)
    im = {k: v.detach().cpu().numpy() for k, v in gpu_img.items()}
    bad = np.abs(im["color"] - ora["color"]).max(0) > 1e-4
    for k in ("depth", "alpha", "nu_map", "median", "T_final"):
        bad |= np.abs(im[k] - ora[k]) > 1e-4
    assert np.all(ora["margins"].min(axis=0)[bad] < 1e-5)
    return int(bad.sum())


def _posed(T, xi):
    rho, phi = np.asarray(xi[:3]), np.asarray(xi[3:])
    th = np.linalg.norm(phi)
    K = np.array([[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]])
    R = np.eye(3) if th == 0 else np.eye(3) + math.sin(th) / th * K + (1 - math.cos(th)) / th ** 2 * K @ K
    out = np.zeros((3, 4))
    out[:, :3] = R @ T[:, :3]
    out[:, 3] = R @ T[:, 3] + rho
    return out


def test_alignment_loss_through_autograd_matches_oracle():
    """L = 0.7 L1 colour + 0.25 L1 depth + 0.25 |D_alpha - D_median| (the
    mapping weights omega_1, omega_3, omega_4 of Sec. 4)."""
    from paper_2403_16095_b300 import Rasterizer, rasterize
    from paper_2403_16095_b300 import _abi as A
    sc, cam, T = synth.tiny_scene()
    T = _posed(np.asarray(T, np.float64), [0.02, -0.01, 0.05, 0.01, 0.02, -0.03]).astype(np.float32).astype(np.float64)
    tc, td = synth.random_targets(cam, 1001 + 81)
    g = to_gpu_gaussians(sc)
    for k in PARAMS:
        getattr(g, k).requires_grad_(True)
    xi = torch.zeros(1, 6, device="cuda", requires_grad=True)
    r = Rasterizer([cam], sc.n, tile=16, mode=A.GS_MODE_FULL)
    out = rasterize(g, xi, poses_gpu(T), r)
    HW = cam.width * cam.height
    loss = (0.7 * (out["color"] - torch.from_numpy(tc[0]).cuda().reshape(-1)).abs().sum()
            + 0.25 * (out["depth"] - torch.from_numpy(td[0]).cuda().reshape(-1)).abs().sum()
            + 0.25 * (out["depth"] - out["median"]).abs().sum()) / HW
    loss.backward()
    og = oracle.grad(f32_scene(sc), cam, T,
                     oracle.LossSpec(0.7, 0.25, 0, 0, 0, tc[0], td[0], w_align=0.25))
    assert abs(float(loss.detach()) - og["loss"]) < 1e-4 * og["loss"]
    n_flip = _n_flip(sc, cam, T, r.frame_images(0))
    assert n_flip <= 3
    for k in PARAMS:
        if k == "nu":
            continue  # no term reaches nu
        _rel(k, getattr(g, k).grad.cpu().numpy(), og[k], n_flip=n_flip)
    _rel("xi", xi.grad[0].cpu().numpy(), og["pose"], elem=1e-4, norm=1e-4)


@pytest.fixture(scope="module")
def window():
    """4 keyframes (k = 4, Sec. 4) of a room on a circle, 160x120, 60k Gaussians."""
    sc = synth.room_scene(60_000, seed=1003)
    cam = synth.Camera(160, 120, 150.0, 150.0, 80.0, 60.0)
    poses = synth.circle_poses(4, seed=1003)
    Ts = [np.asarray(T, np.float32).astype(np.float64) for T in poses]
    tgts = [synth.random_targets(cam, 1003 + 20 + f, depth_range=(0.5, 4.0)) for f in range(4)]
    return sc, cam, Ts, [t[0][0] for t in tgts], [t[1][0] for t in tgts]


def test_keyframe_window_in_one_launch_matches_per_frame_oracle(window):
    """f3: the FULL backward over 4 keyframes in one launch gives parameter
    gradients equal to the sum of the per-frame oracle gradients and one pose
    gradient per keyframe."""
    from paper_2403_16095_b300 import Rasterizer
    from paper_2403_16095_b300 import _abi as A
    sc, cam, Ts, tcs, tds = window
    g = to_gpu_gaussians(sc)
    F = len(Ts)
    r = Rasterizer([cam] * F, sc.n, tile=16, mode=A.GS_MODE_FULL)
    Tt = poses_gpu(np.stack(Ts))
    obs = torch.from_numpy(np.stack(tds)).cuda().reshape(-1)
    r.render(g, Tt, obs)
    loss = dict(w_color=0.7, w_depth=0.25, target_color=torch.from_numpy(np.stack(tcs)).cuda().reshape(-1),
                target_depth=obs)
    grads = {k: torch.empty_like(getattr(g, k)) for k in PARAMS}
    r.backward(obs_depth=obs, loss=loss, g=g, T_cw=Tt, grads=grads)
    torch.cuda.synchronize()
    assert r.read_status()[0] == 0
    s64 = f32_scene(sc)
    want = {k: 0.0 for k in PARAMS}
    for f in range(F):
        og = oracle.grad(s64, cam, Ts[f], oracle.LossSpec(0.7, 0.25, 0, 0, 0, tcs[f], tds[f]))
        for k in PARAMS:
            want[k] = want[k] + og[k]
        _rel(f"pose[{f}]", r.pose_grad[f].cpu().numpy(), og["pose"], elem=1e-4, norm=1e-4)
    for k in PARAMS:
        if k == "nu":
            assert float(grads[k].abs().max()) == 0.0
            continue
        _rel(k, grads[k].cpu().numpy(), want[k], elem=1e-3, norm=1e-4)


def test_gpu_gradient_matches_oracle_central_differences():
    """North-star check (3): the autograd gradient on the GPU against central
    differences (h = 1e-4) of the FP64 oracle loss, on every parameter of sampled
    Gaussians whose pixel decisions do not change within +-h. The tolerance is
    FP32 gradient accuracy (relative 2e-3 of the largest element)."""
    from paper_2403_16095_b300 import Rasterizer, rasterize
    from paper_2403_16095_b300 import _abi as A
    sc32, cam, T = synth.fd_scene()
    sc32 = synth.Scene(*(np.asarray(getattr(sc32, k), np.float32) for k in PARAMS))
    sc = f32_scene(sc32)
    tc, td = synth.random_targets(cam, 1100 + 9, depth_range=(2, 4))
    g = to_gpu_gaussians(sc32)
    for k in PARAMS:
        getattr(g, k).requires_grad_(True)
    xi = torch.zeros(1, 6, device="cuda", requires_grad=True)
    r = Rasterizer([cam], sc.n, tile=16, mode=A.GS_MODE_FULL)
    out = rasterize(g, xi, poses_gpu(T), r)
    HW = cam.width * cam.height
    loss = ((out["color"] - torch.from_numpy(tc[0]).cuda().reshape(-1)).abs().sum()
            + (out["depth"] - torch.from_numpy(td[0]).cuda().reshape(-1)).abs().sum()) / HW
    loss.backward()
    L = oracle.LossSpec(1.0, 1.0, 0, 0, 0, tc[0], td[0])
    _, h0 = oracle.loss_value(sc, cam, T, L)
    h = 1e-4
    rng = np.random.default_rng(0)
    checked = 0
    for i in rng.choice(sc.n, 16, replace=False):
        for field, dim in (("means", 3), ("log_scales", 3), ("quats", 4), ("opacity_logit", 1), ("colors", 3)):
            arr = getattr(sc, field)
            gpu = getattr(g, field).grad.cpu().numpy().astype(np.float64)
            scale = np.abs(gpu).max()
            for c in range(dim):
                idx = (i, c) if arr.ndim == 2 else (i,)
                old = arr[idx]
                arr[idx] = old + h
                vp, hp = oracle.loss_value(sc, cam, T, L)
                arr[idx] = old - h
                vm, hm = oracle.loss_value(sc, cam, T, L)
                arr[idx] = old
                if hp != h0 or hm != h0:
                    continue
                fd = (vp - vm) / (2 * h)
                assert abs(gpu[idx] - fd) <= 2e-3 * scale, (field, i, c, gpu[idx], fd)
                checked += 1
    assert checked >= 100


def test_autotuned_uneven_batch_is_tile_invariant():
    """Config-4 machinery on a small uneven batch (3 resolutions, 5 frames): the
    autotuner's pick is the fastest of its own timings, and every tile size gives
    bit-identical images and the same FULL-mode gradients (up to the order of the
    FP32 atomic sums)."""
    from paper_2403_16095_b300 import Rasterizer, autotune_tile
    from paper_2403_16095_b300 import _abi as A
    sc = synth.room_scene(40_000, seed=1006)
    cams = [synth.Camera(96, 64, 90.0, 90.0, 48.0, 32.0), synth.Camera(160, 120, 150.0, 150.0, 80.0, 60.0),
            synth.Camera(200, 113, 187.5, 187.5, 100.0, 56.5)] + [synth.Camera(160, 120, 150.0, 150.0, 80.0, 60.0)] * 2
    Ts = np.stack([np.asarray(T, np.float32) for T in synth.circle_poses(5, seed=1006)])
    g = to_gpu_gaussians(sc)
    Tt = poses_gpu(Ts)
    tg = [synth.random_targets(c, 1006 + 10 + f, depth_range=(0.5, 4.0)) for f, c in enumerate(cams)]
    tc = torch.from_numpy(np.concatenate([t[0].reshape(-1) for t in tg])).cuda()
    td = torch.from_numpy(np.concatenate([t[1].reshape(-1) for t in tg])).cuda()
    loss = dict(w_color=0.7, w_depth=0.25, w_unc=0.15, w_align=0.25, target_color=tc, target_depth=td)
    best, times = autotune_tile(cams, g, Tt, td, mode=A.GS_MODE_FULL, loss=loss)
    assert best == min(times, key=times.get) and set(times) == {8, 16, 32}
    imgs, grads = {}, {}
    for t in (8, 16, 32):
        r = Rasterizer(cams, sc.n, tile=t, mode=A.GS_MODE_FULL)
        r.render(g, Tt, td)
        gr = {k: torch.empty_like(getattr(g, k)) for k in PARAMS}
        r.backward(obs_depth=td, loss=loss, g=g, T_cw=Tt, grads=gr)
        torch.cuda.synchronize()
        assert r.read_status()[0] == 0
        imgs[t] = {k: v.clone() for k, v in r.img.items()}
        grads[t] = {k: v.cpu().numpy() for k, v in gr.items()}
        grads[t]["pose"] = r.pose_grad.cpu().numpy()
    for t in (8, 32):
        for k in ("color", "depth", "alpha", "unc", "median", "T_final", "n_contrib"):
            assert torch.equal(imgs[t][k], imgs[16][k]), (t, k)
        for k in list(PARAMS[:-1]) + ["pose"]:
            a, b = grads[t][k], grads[16][k]
            assert np.abs(a - b).max() <= 1e-5 * np.abs(b).max(), (t, k)


def test_maximum_frame_count_in_one_launch():
    """The largest batch one call takes (64 frames, three image sizes, each its
    own pose): per-frame images, per-frame pose gradients and the parameter
    gradients summed over the frames equal 64 separate oracle evaluations."""
    from paper_2403_16095_b300 import Rasterizer
    from paper_2403_16095_b300 import _abi as A
    F = A.GS_MAX_FRAMES
    sc, _, _ = synth.tiny_scene(n=600, seed=1301)
    sizes = [(40, 30, 30.0), (33, 21, 25.0), (24, 40, 35.0)]
    cams = [synth.Camera(w, h, fo, fo, w / 2, h / 2) for w, h, fo in (sizes[f % 3] for f in range(F))]
    rng = np.random.default_rng(1301)
    T0 = np.c_[np.eye(3), np.zeros(3)]
    Ts = [_posed(T0, np.r_[rng.uniform(-0.1, 0.1, 3), rng.uniform(-0.05, 0.05, 3)]).astype(np.float32)
          .astype(np.float64) for _ in range(F)]
    tgts = [synth.random_targets(cams[f], 1301 + 1 + f) for f in range(F)]
    tc = np.concatenate([t[0][0].reshape(-1) for t in tgts])
    td = np.concatenate([t[1][0].reshape(-1) for t in tgts])
    g = to_gpu_gaussians(sc)
    r = Rasterizer(cams, sc.n, tile=16, mode=A.GS_MODE_FULL)
    Tt = poses_gpu(np.stack(Ts))
    obs = torch.from_numpy(td).cuda()
    r.render(g, Tt, obs)
    loss = dict(w_color=0.7, w_depth=0.25, target_color=torch.from_numpy(tc).cuda(), target_depth=obs)
    grads = {k: torch.empty_like(getattr(g, k)) for k in PARAMS}
    r.backward(obs_depth=obs, loss=loss, g=g, T_cw=Tt, grads=grads)
    torch.cuda.synchronize()
    assert r.read_status()[0] == 0
    s64 = f32_scene(sc)
    want = {k: 0.0 for k in PARAMS}
    n_flip = 0
    for f in range(F):
        n_flip += _n_flip(sc, cams[f], Ts[f], r.frame_images(f))
        og = oracle.grad(s64, cams[f], Ts[f], oracle.LossSpec(0.7, 0.25, 0, 0, 0, tgts[f][0][0], tgts[f][1][0]))
        for k in PARAMS:
            want[k] = want[k] + og[k]
        _rel(f"pose[{f}]", r.pose_grad[f].cpu().numpy(), og["pose"], elem=1e-4, norm=1e-4)
    assert n_flip <= 8
    for k in PARAMS:
        if k == "nu":
            assert float(grads[k].abs().max()) == 0.0
            continue
        _rel(k, grads[k].cpu().numpy(), want[k], elem=1e-3, norm=1e-4, n_flip=n_flip)
