"""Tracking (Sec. 3.4, Eq. 19-20) on the GPU, and full-size parity at the
640x480 / 300,000-Gaussian tracking workload in the launch configuration the
benchmark times (tile 16, POSE mode, fused uncertainty-weighted L1 loss)."""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_util import IMG_TOL, at_decision_margin, f32_scene, image_mismatch, poses_gpu, to_gpu_gaussians

pytestmark = pytest.mark.gpu


def _pose_err(Ta, Tb):
    Ta, Tb = np.asarray(Ta, float), np.asarray(Tb, float)
    ca = -Ta[:, :3].T @ Ta[:, 3]
    cb = -Tb[:, :3].T @ Tb[:, 3]
    dR = Ta[:, :3] @ Tb[:, :3].T
    ang = math.degrees(math.acos(max(-1.0, min(1.0, (np.trace(dR) - 1) / 2))))
    return float(np.linalg.norm(ca - cb)), ang


@pytest.fixture(scope="module")
def room_small():
    sc = synth.room_scene(80_000, seed=1302)
    cam = synth.Camera(320, 240, 300.0, 300.0, 160.0, 120.0)
    poses = synth.room_track_poses(3, seed=1302)
    return sc, cam, poses


def _targets(sc, cam, T):
    """Target RGB-D rendered at the ground-truth pose (an input of the tracking
    test, whose check is convergence towards that pose)."""
    from paper_2403_16095_b300 import Rasterizer
    from paper_2403_16095_b300 import _abi as A
    r = Rasterizer([cam], sc.n, tile=16, mode=A.GS_MODE_FWD)
    r.render(to_gpu_gaussians(sc), poses_gpu(T))
    im = r.frame_images(0)
    return im["color"].clone(), im["depth"].clone()


@pytest.mark.parametrize("graph", [False, True])
def test_tracking_converges_towards_ground_truth(room_small, graph):
    from paper_2403_16095_b300 import Tracker
    sc, cam, poses = room_small
    g = to_gpu_gaussians(sc)
    T_gt = poses[1]
    tcol, tdep = _targets(sc, cam, T_gt)
    T0 = synth.jitter_pose(T_gt, seed=77, trans=0.02, rot_deg=1.0)
    tr = Tracker(g, cam, iters=30, graph=graph)
    tr.prepare(tcol, tdep, torch.from_numpy(T0))
    T = tr.track(tcol, tdep, torch.from_numpy(T0)).cpu().numpy()
    e0 = _pose_err(T0, T_gt)
    e1 = _pose_err(T, T_gt)
    print("start (m, deg)", e0, "end", e1)
    # 30 Adam steps at lr {0.0015 rad, 0.00215 m} from a 2 cm / 1 degree jitter
    assert e1[0] < 0.8 * e0[0] and e1[1] < 0.6 * e0[1]


def test_graph_replay_equals_eager(room_small):
    from paper_2403_16095_b300 import Tracker
    sc, cam, poses = room_small
    g = to_gpu_gaussians(sc)
    tcol, tdep = _targets(sc, cam, poses[0])
    T0 = torch.from_numpy(synth.jitter_pose(poses[0], seed=5))
    out = []
    for graph in (False, True):
        tr = Tracker(g, cam, iters=10, graph=graph)
        tr.prepare(tcol, tdep, T0)
        out.append(tr.track(tcol, tdep, T0))
    assert torch.equal(out[0], out[1])


# ------------------------------------------------------------- full size
@pytest.fixture(scope="module")
def track_full():
    w = synth.workload("track")
    sc, cam, poses = w["scene"], w["cams"][0], w["poses"]
    T = np.asarray(synth.jitter_pose(poses[0], seed=1002 + 1), np.float32).astype(np.float64)
    # targets are the oracle's own render at the ground-truth pose
    ref = oracle.render(f32_scene(sc), cam, np.asarray(poses[0], np.float32).astype(np.float64))
    return sc, cam, T, ref["color"].astype(np.float32), ref["depth"].astype(np.float32)


def test_full_size_forward_matches_oracle(track_full):
    from paper_2403_16095_b300 import Rasterizer
    from paper_2403_16095_b300 import _abi as A
    sc, cam, T, tc, td = track_full
    r = Rasterizer([cam], sc.n, tile=16, mode=A.GS_MODE_POSE)
    obs = torch.from_numpy(td).cuda().reshape(-1)
    r.render(to_gpu_gaussians(sc), poses_gpu(T), obs)
    torch.cuda.synchronize()
    im = {k: v.cpu().numpy() for k, v in r.frame_images(0).items()}
    ora = oracle.render(f32_scene(sc), cam, T, obs_depth=td)
    # every channel, U included, within IMG_TOL absolute (U reaches ~4 m^2 here;
    # its FP32 error away from decision margins measured 1e-5)
    bad = image_mismatch(im, ora)
    frac = bad.mean()
    print("pixels beyond", IMG_TOL, ":", int(bad.sum()), "of", bad.size)
    assert frac < 2e-3
    assert np.all(at_decision_margin(ora)[bad])


def test_full_size_pose_gradient_matches_oracle(track_full):
    from paper_2403_16095_b300 import Rasterizer
    from paper_2403_16095_b300 import _abi as A
    sc, cam, T, tc, td = track_full
    r = Rasterizer([cam], sc.n, tile=16, mode=A.GS_MODE_POSE)
    obs = torch.from_numpy(td).cuda().reshape(-1)
    r.render(to_gpu_gaussians(sc), poses_gpu(T), obs)
    loss = dict(w_color=0.2, w_depth=1.0, unc_tau=0.025, target_color=torch.from_numpy(tc).cuda().reshape(-1),
                target_depth=obs)
    r.backward(obs_depth=obs, loss=loss)
    r.reduce_pose()
    torch.cuda.synchronize()
    og = oracle.grad(f32_scene(sc), cam, T, oracle.LossSpec(0.2, 1.0, 0.0, 0.0, 0.025, tc, td))
    got = r.pose_grad[0].cpu().numpy()
    rel = np.abs(got - og["pose"]).max() / np.abs(og["pose"]).max()
    print("full-size pose gradient", got, og["pose"], rel)
    assert rel < 5e-5  # measured 5.3e-6 on a B300


def test_fused_tracking_pass_equals_forward_then_backward(track_full):
    """gs_render_fwd_bwd_pose (one launch per tile) reproduces gs_render_fwd +
    gs_render_bwd (POSE, tracking loss) bit for bit: the tracking channels and
    the FP64 pose gradient, at 640x480 / 300k in the benchmark's configuration."""
    from paper_2403_16095_b300 import Rasterizer
    from paper_2403_16095_b300 import _abi as A
    sc, cam, T, tc, td = track_full
    obs = torch.from_numpy(td).cuda().reshape(-1)
    loss = dict(w_color=0.2, w_depth=1.0, unc_tau=0.025, target_color=torch.from_numpy(tc).cuda().reshape(-1),
                target_depth=obs)
    res = []
    for fused in (False, True):
        r = Rasterizer([cam], sc.n, tile=16, mode=A.GS_MODE_POSE, channels="track")
        r.render(to_gpu_gaussians(sc), poses_gpu(T), obs)
        for k in r.img:
            r.img[k].fill_(-1 if r.img[k].dtype == torch.int32 else float("nan"))
        r.pose_grad.zero_()
        if fused:
            r.fwd_bwd_pose(loss, images=True)
        else:
            r.forward(obs)
            r.backward(obs_depth=obs, loss=loss)
        torch.cuda.synchronize()
        assert r.read_status()[0] == 0
        res.append(({k: v.clone() for k, v in r.img.items()}, r.pose_grad.clone()))
    for k in res[0][0]:
        assert torch.equal(res[0][0][k], res[1][0][k]), k
    assert torch.equal(res[0][1], res[1][1])
    # losses beyond colour and depth are refused by the fused pass
    with pytest.raises(A.GsError):
        r.fwd_bwd_pose(dict(loss, w_align=0.1))


def test_fused_tracking_pass_long_lists_equal_forward_then_backward():
    """Long tile lists, walked in several staging batches and restaged for the
    backward: 12,000 Gaussians over the 12 tiles of a 64x48 image (1,000 per
    tile). The tracking pass's channels and FP64 pose gradient equal
    gs_render_fwd + gs_render_bwd bit for bit."""
    from paper_2403_16095_b300 import Rasterizer
    from paper_2403_16095_b300 import _abi as A
    sc = synth.room_scene(12_000, seed=1309)
    cam = synth.Camera(64, 48, 60.0, 60.0, 32.0, 24.0)
    poses = synth.room_track_poses(2, seed=1309)
    T_gt = poses[0]
    g = to_gpu_gaussians(sc)
    r0 = Rasterizer([cam], sc.n, tile=16, mode=A.GS_MODE_FWD)
    r0.render(g, poses_gpu(T_gt))
    tc, td = r0.img["color"].clone(), r0.img["depth"].clone()
    assert sc.n >= 800 * r0.n_tiles
    T = synth.jitter_pose(T_gt, seed=7)
    loss = dict(w_color=0.2, w_depth=1.0, unc_tau=0.025, target_color=tc, target_depth=td)
    res = []
    for fused in (False, True):
        r = Rasterizer([cam], sc.n, tile=16, mode=A.GS_MODE_POSE, channels="track")
        r.render(g, poses_gpu(T), td)
        for k in r.img:
            r.img[k].fill_(-1 if r.img[k].dtype == torch.int32 else float("nan"))
        r.pose_grad.zero_()
        if fused:
            r.fwd_bwd_pose(loss, images=True)
        else:
            r.forward(td)
            r.backward(obs_depth=td, loss=loss)
        torch.cuda.synchronize()
        code, P = r.read_status()
        assert code == 0 and P > 10 * r.n_tiles
        res.append(({k: v.clone() for k, v in r.img.items()}, r.pose_grad.clone()))
    for k in res[0][0]:
        assert torch.equal(res[0][0][k], res[1][0][k]), k
    assert torch.equal(res[0][1], res[1][1])
    assert float(res[1][1].abs().max()) > 0


@pytest.mark.parametrize("n", [255, 256, 257, 511, 512, 513])
def test_fused_tracking_pass_at_staging_batch_boundaries(n):
    """Every tile list exactly n entries long, around one and two 256-entry
    staging batches: n broad, faint Gaussians in front of a 64x48 camera, each
    covering all 12 tiles and blended by the central pixels without saturating
    them. A list of one batch is walked back by each warp on its own; a longer
    one is restaged batch by batch. Both equal gs_render_fwd + gs_render_bwd
    bit for bit (tracking channels and FP64 pose gradient)."""
    from paper_2403_16095_b300 import Rasterizer
    from paper_2403_16095_b300 import _abi as A
    rng = np.random.default_rng(1400 + n)
    z = rng.uniform(2.5, 3.5, n)
    means = np.stack([rng.uniform(-0.05, 0.05, n) * z, rng.uniform(-0.05, 0.05, n) * z, z], 1)
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    sc = synth.Scene(means.astype(np.float32), np.full((n, 3), math.log(0.8), np.float32), q.astype(np.float32),
                     rng.normal(-4.6, 0.15, n).astype(np.float32), rng.uniform(0, 1, (n, 3)).astype(np.float32),
                     rng.uniform(0, 0.1, n).astype(np.float32))
    cam = synth.Camera(64, 48, 60.0, 60.0, 32.0, 24.0)
    T = synth.jitter_pose(np.c_[np.eye(3), np.zeros(3)], seed=n)
    g = to_gpu_gaussians(sc)
    tc = torch.rand(3 * 64 * 48, device="cuda", generator=torch.Generator("cuda").manual_seed(n))
    td = torch.rand(64 * 48, device="cuda", generator=torch.Generator("cuda").manual_seed(n + 1)) + 2.5
    loss = dict(w_color=0.2, w_depth=1.0, unc_tau=0.025, target_color=tc, target_depth=td)
    res = []
    for fused in (False, True):
        r = Rasterizer([cam], n, tile=16, mode=A.GS_MODE_POSE, channels="track")
        r.render(g, poses_gpu(T), td)
        lens = (r.ranges[1::2] - r.ranges[0::2]).cpu()
        assert bool(torch.all(lens == n)), lens
        for k in r.img:
            r.img[k].fill_(-1 if r.img[k].dtype == torch.int32 else float("nan"))
        r.pose_grad.zero_()
        if fused:
            r.fwd_bwd_pose(loss, images=True)
        else:
            r.forward(td)
            r.backward(obs_depth=td, loss=loss)
        torch.cuda.synchronize()
        assert r.read_status()[0] == 0
        res.append(({k: v.clone() for k, v in r.img.items()}, r.pose_grad.clone()))
    for k in res[0][0]:
        assert torch.equal(res[0][0][k], res[1][0][k]), k
    assert torch.equal(res[0][1], res[1][1])
    # the central pixel blends every entry of its tile (tile 6 of the 4x3
    # grid), so its warps walk the whole list back
    assert int(res[1][0]["n_last"][24 * 64 + 32]) == int(r.ranges[2 * 6 + 1])
    assert float(res[1][0]["T_final"].min()) > 1e-3
    assert float(res[1][1].abs().max()) > 0


def test_tracker_fused_equals_unfused(room_small):
    from paper_2403_16095_b300 import Tracker
    sc, cam, poses = room_small
    g = to_gpu_gaussians(sc)
    tcol, tdep = _targets(sc, cam, poses[0])
    T0 = torch.from_numpy(synth.jitter_pose(poses[0], seed=6))
    out = []
    for fused in (False, True):
        tr = Tracker(g, cam, iters=10, graph=True, fused=fused)
        tr.prepare(tcol, tdep, T0)
        out.append(tr.track(tcol, tdep, T0))
    assert torch.equal(out[0], out[1])


def test_tracking_pass_two_frames_with_adam_equals_separate_calls(room_small):
    """The tracking pass over a batch of two frames (different poses, one launch)
    gives each frame the same pose gradient and the same Adam update as the
    separate forward, backward and gs_pose_adam_step calls."""
    from paper_2403_16095_b300 import Rasterizer
    from paper_2403_16095_b300 import _abi as A
    from paper_2403_16095_b300.raster import pose_state
    sc, cam, poses = room_small
    g = to_gpu_gaussians(sc)
    tgt = [_targets(sc, cam, poses[f]) for f in (0, 2)]
    tc = torch.cat([t[0].reshape(-1) for t in tgt])
    td = torch.cat([t[1].reshape(-1) for t in tgt])
    T0 = np.stack([synth.jitter_pose(poses[f], seed=40 + f) for f in (0, 2)])
    loss = dict(w_color=0.2, w_depth=1.0, unc_tau=0.025, target_color=tc, target_depth=td)
    adam = A.gs_adam(0.0015, 0.00215, 0.9, 0.999, 1e-8)
    out = []
    for fused in (False, True):
        r = Rasterizer([cam, cam], sc.n, tile=16, mode=A.GS_MODE_POSE, channels="track")
        Tt = poses_gpu(T0).clone()
        state = pose_state(torch.from_numpy(T0).cuda()).contiguous()
        r.render(g, Tt, td)
        if fused:
            r.fwd_bwd_pose(loss, adam_state=state, adam=adam, T_cw=Tt)
        else:
            r.forward(td)
            r.backward(obs_depth=td, loss=loss)
            A.gs_pose_adam_step(state, r.pose_grad, Tt, 2, adam, r.status)
        torch.cuda.synchronize()
        assert r.read_status()[0] == 0
        out.append((r.pose_grad.clone(), state.clone(), Tt.clone()))
    for a, b in zip(out[0], out[1]):
        assert torch.equal(a, b)
    assert float(out[0][0][0].abs().max()) > 0 and float(out[0][0][1].abs().max()) > 0


@pytest.mark.parametrize("fused", [True, False])
def test_tracker_recovers_from_pair_overflow(room_small, fused):
    """A tracker whose pair buffer is far too small: the first attempt overflows
    (device status, every later kernel of the frame no-ops), the buffer grows,
    the graph is recaptured and the frame is tracked again from its start pose;
    the result equals that of a tracker sized correctly up front."""
    from paper_2403_16095_b300 import Tracker
    sc, cam, poses = room_small
    g = to_gpu_gaussians(sc)
    tcol, tdep = _targets(sc, cam, poses[1])
    T0 = torch.from_numpy(synth.jitter_pose(poses[1], seed=9))
    small = Tracker(g, cam, iters=10, graph=True, fused=fused, capacity=64)
    got = small.track(tcol, tdep, T0)
    assert small.rast.capacity > 64
    ref = Tracker(g, cam, iters=10, graph=True, fused=fused)
    ref.prepare(tcol, tdep, T0)
    assert torch.equal(got, ref.track(tcol, tdep, T0))


def _host_frames(sc, cam, poses, seeds):
    """Pinned host RGB-D targets and start poses of a few frames."""
    hc, hd, hT = [], [], []
    for k, seed in enumerate(seeds):
        tcol, tdep = _targets(sc, cam, poses[k % len(poses)])
        hc.append(tcol.cpu().pin_memory())
        hd.append(tdep.cpu().pin_memory())
        hT.append(torch.from_numpy(synth.jitter_pose(poses[k % len(poses)], seed=seed)).pin_memory())
    return hc, hd, hT


def test_streaming_submit_equals_track_host(room_small):
    """Tracker.submit/drain (uploads on a copy stream into two staging buffers,
    overlapped with the tracking of the previous frame) gives, frame by frame,
    the same poses as the synchronous track_host; six frames reuse each staging
    buffer three times."""
    from paper_2403_16095_b300 import Tracker
    sc, cam, poses = room_small
    g = to_gpu_gaussians(sc)
    hc, hd, hT = _host_frames(sc, cam, poses, seeds=[21, 22, 23, 24, 25, 26])
    tr = Tracker(g, cam, iters=10, graph=True)
    tr.prepare(hc[0].cuda(), hd[0].cuda(), hT[0])
    ref = [tr.track_host(hc[k], hd[k], hT[k]) for k in range(6)]
    outs = [torch.full((3, 4), float("nan"), dtype=torch.float64).pin_memory() for _ in range(6)]
    for k in range(6):
        tr.submit(hc[k], hd[k], hT[k], outs[k])
    assert tr.drain() == 6
    for k in range(6):
        assert torch.equal(outs[k], ref[k]), k
    assert not torch.equal(ref[0], ref[1])


def test_streaming_redoes_frames_that_overflowed(room_small):
    """Frames submitted to a tracker whose pair buffer is far too small all
    overflow on the device; drain() tracks each of them again synchronously
    (growing the buffer) and their poses equal a correctly sized tracker's."""
    from paper_2403_16095_b300 import Tracker
    sc, cam, poses = room_small
    g = to_gpu_gaussians(sc)
    hc, hd, hT = _host_frames(sc, cam, poses, seeds=[31, 32, 33])
    small = Tracker(g, cam, iters=10, graph=True, capacity=64)
    small.set_frame(hc[0].cuda(), hd[0].cuda(), hT[0])
    small._capture()
    outs = [torch.empty(3, 4, dtype=torch.float64).pin_memory() for _ in range(3)]
    for k in range(3):
        small.submit(hc[k], hd[k], hT[k], outs[k])
    small.drain()
    assert small.rast.capacity > 64
    ref = Tracker(g, cam, iters=10, graph=True)
    ref.prepare(hc[0].cuda(), hd[0].cuda(), hT[0])
    for k in range(3):
        assert torch.equal(outs[k], ref.track_host(hc[k], hd[k], hT[k])), k


def test_tracking_pass_with_every_gaussian_culled():
    """All Gaussians behind the camera: the tracking pass renders nothing, the
    pose gradient is exactly zero, and the Adam step leaves the pose unchanged."""
    from paper_2403_16095_b300 import Rasterizer
    from paper_2403_16095_b300 import _abi as A
    from paper_2403_16095_b300.raster import pose_state
    sc, _, _ = synth.tiny_scene(n=200, seed=1205)
    behind = synth.Scene(sc.means * np.float32([1, 1, -1]), sc.log_scales, sc.quats, sc.opacity_logit, sc.colors,
                         sc.nu)
    cam = synth.Camera(64, 48, 50.0, 50.0, 32.0, 24.0)
    T = np.c_[np.eye(3), np.zeros(3)]
    r = Rasterizer([cam], behind.n, tile=16, mode=A.GS_MODE_POSE, channels="track")
    Tt = poses_gpu(T).clone()
    r.render(to_gpu_gaussians(behind), Tt)
    tc = torch.rand(3 * 64 * 48, device="cuda")
    td = torch.rand(64 * 48, device="cuda") + 1.0
    state = pose_state(torch.from_numpy(T).cuda()).contiguous()
    r.fwd_bwd_pose(dict(w_color=0.2, w_depth=1.0, unc_tau=0.025, target_color=tc, target_depth=td), images=True,
                   adam_state=state, adam=A.gs_adam(0.0015, 0.00215, 0.9, 0.999, 1e-8), T_cw=Tt)
    torch.cuda.synchronize()
    assert r.read_status() == (0, 0)
    assert float(r.pose_grad.abs().max()) == 0.0
    assert torch.equal(Tt, poses_gpu(T))
    assert bool(torch.all(r.img["T_final"] == 1.0)) and float(r.img["color"].abs().max()) == 0.0


def test_tracking_an_empty_map_keeps_the_start_pose(room_small):
    """A map with no Gaussians: every tile list is empty, the pose gradient is
    exactly zero, and the Adam steps leave the start pose unchanged."""
    from paper_2403_16095_b300 import Gaussians, Tracker
    sc, cam, poses = room_small
    tcol, tdep = _targets(sc, cam, poses[0])
    e = torch.zeros(0, device="cuda")
    g = Gaussians(e.view(0, 3), e.view(0, 3), torch.zeros(0, 4, device="cuda"), e, e.view(0, 3), e)
    T0 = torch.from_numpy(synth.jitter_pose(poses[0], seed=41))
    tr = Tracker(g, cam, iters=5, graph=True, capacity=4096)
    tr.prepare(tcol, tdep, T0)
    T = tr.track(tcol, tdep, T0).cpu()
    assert torch.allclose(T, T0.to(T.dtype), rtol=0, atol=1e-12)
