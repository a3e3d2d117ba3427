"""16-bit Gaussian storage on the GPU (per-chunk fixed-point means, BF16
attributes) against the oracle's model of it, and the rasterizer on that
storage against the FP64 oracle of the Gaussians it represents.

* spatial order, chunk boxes and packed bits: bit-exact (integer work, and FP32
  decisions taken with the same round-to-nearest operations on both sides);
* projection from packed storage == FP32 projection of the decoded values, bit
  for bit (the decode is exact and the arithmetic is the same);
* the 5M-Gaussian 1200x680 workload rendered from packed storage against the
  oracle on sampled pixels, with the storage error itself reported;
* tracking from packed storage converges like tracking from FP32."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_util import f32_scene, poses_gpu, to_gpu_gaussians

pytestmark = pytest.mark.gpu


def test_spatial_order_and_packing_bit_exact():
    from paper_2403_16095_b300 import pack_bf16
    for n, seed in ((200_000, 1005), (1000, 7), (257, 8)):
        sc = synth.room_scene(n, seed=seed) if n > 1000 else synth.tiny_scene(n, seed=seed)[0]
        g = to_gpu_gaussians(sc)
        pk = pack_bf16(g, spatial=True)
        torch.cuda.synchronize()
        perm = oracle.spatial_order(np.asarray(sc.means, np.float32))
        assert np.array_equal(pk.perm.cpu().numpy(), perm)
        anchors, packed = oracle.pack_bf16(f32_scene(sc), perm)
        assert np.array_equal(pk.anchors.cpu().numpy().view(np.uint32), anchors.view(np.uint32))
        assert np.array_equal(pk.packed.cpu().numpy().view(np.uint16), packed)
    # without a permutation the source order is kept
    pk = pack_bf16(g, spatial=False)
    anchors, packed = oracle.pack_bf16(f32_scene(sc), None)
    assert np.array_equal(pk.packed.cpu().numpy().view(np.uint16), packed)


def test_projection_from_packed_equals_fp32_projection_of_decoded():
    from paper_2403_16095_b300 import Rasterizer, pack_bf16
    from paper_2403_16095_b300 import _abi as A
    sc = synth.room_scene(300_000, seed=1002)
    cam = synth.Camera(640, 480, 600.0, 600.0, 320.0, 240.0)
    T = np.asarray(synth.room_track_poses(10, seed=1002)[3], np.float32)
    pk = pack_bf16(to_gpu_gaussians(sc), spatial=True)
    dec = oracle.unpack_bf16(pk.anchors.cpu().numpy(), pk.packed.cpu().numpy().view(np.uint16))
    for mode in (A.GS_MODE_FWD, A.GS_MODE_POSE):
        ra = Rasterizer([cam], sc.n, tile=16, mode=mode)
        rb = Rasterizer([cam], sc.n, tile=16, mode=mode)
        ra.project(pk, poses_gpu(T))
        rb.project(to_gpu_gaussians(dec), poses_gpu(T))
        torch.cuda.synchronize()
        assert torch.equal(ra.touched, rb.touched)
        ia, ib = ra.rec.view(-1, 16).view(torch.int32), rb.rec.view(-1, 16).view(torch.int32)
        vis = ra.touched > 0  # a culled record holds only its (empty) rect
        assert torch.equal(ia[vis], ib[vis]) and torch.equal(ia[:, 12:], ib[:, 12:])
        if mode == A.GS_MODE_POSE:
            ja, jb = ra.jac.view(-1, 36).view(torch.int32), rb.jac.view(-1, 36).view(torch.int32)
            assert torch.equal(ja[vis], jb[vis])
    with pytest.raises(A.GsError):
        Rasterizer([cam], sc.n, tile=16, mode=A.GS_MODE_FULL).project(pk, poses_gpu(T))


@pytest.fixture(scope="module")
def precision():
    w = synth.workload("precision")  # 5M Gaussians, 1200x680, 100 poses
    return w["scene"], w["cams"][0], w["poses"]


def test_precision_workload_render_matches_oracle_and_storage_error(precision):
    """Frames 0, 9, 19, ..., 99 of the 5M / 1200x680 workload rendered from
    packed storage: 256 sampled pixels per frame against the oracle of the
    decoded Gaussians (FP32 tolerance 1e-4, decision-margin pixels excepted),
    and the image change caused by the storage itself (FP32 vs packed)."""
    from paper_2403_16095_b300 import Rasterizer, pack_bf16
    from paper_2403_16095_b300 import _abi as A
    sc, cam, poses = precision
    g32 = to_gpu_gaussians(sc)
    pk = pack_bf16(g32, spatial=True)
    dec = oracle.unpack_bf16(pk.anchors.cpu().numpy(), pk.packed.cpu().numpy().view(np.uint16))
    m_err = np.abs(dec.means - np.asarray(sc.means, np.float32)[pk.perm.cpu().numpy()]).max()
    print(f"stored mean error max {m_err * 1e3:.4f} mm")
    assert m_err < 1e-4
    rng = np.random.default_rng(1005)
    HW = cam.width * cam.height
    for f in [0] + list(range(9, 100, 10)):
        T = np.asarray(poses[f], np.float32).astype(np.float64)
        rp = Rasterizer([cam], sc.n, tile=16, mode=A.GS_MODE_FWD)
        rp.render(pk, poses_gpu(T))
        rf = Rasterizer([cam], sc.n, tile=16, mode=A.GS_MODE_FWD)
        rf.render(g32, poses_gpu(T))
        torch.cuda.synchronize()
        ip = {k: v.cpu().numpy() for k, v in rp.frame_images(0).items()}
        i32 = {k: v.cpu().numpy() for k, v in rf.frame_images(0).items()}
        pix = rng.choice(HW, 256, replace=False)
        ora = oracle.render_pixels(dec, cam, T, pix)
        bad = np.zeros(len(pix), bool)
        for k in ("color", "depth", "alpha", "nu_map", "T_final"):
            got = ip[k].reshape(3, -1)[:, pix] if k == "color" else ip[k].reshape(-1)[pix]
            e = np.abs(got - ora[k])
            bad |= (e.max(0) if k == "color" else e) > 1e-4
        # every differing pixel sits at an FP32/FP64 decision margin; with 5M
        # Gaussians a pixel walks hundreds of entries, so some land near q = 9 or
        # alpha = 1/255: the count is reported (bounded loosely)
        assert np.all(ora["margins"].min(0)[bad] < 1e-4), f"frame {f}: mismatch away from a decision margin"
        assert bad.sum() <= 0.05 * len(pix)
        dc = np.abs(ip["color"] - i32["color"])
        dd = np.abs(ip["depth"] - i32["depth"])
        print(f"frame {f}: sampled-pixel flips {int(bad.sum())}; storage error colour mean {dc.mean():.2e} "
              f"max {dc.max():.2e}, depth mean {dd.mean():.2e} m")
        assert dc.mean() < 5e-3 and dd.mean() < 5e-3


def test_tracking_from_packed_storage_converges():
    """Sec. 3.4 tracking with the Gaussians in 16-bit storage: 30 iterations from a
    2 cm / 1 deg perturbed start (targets rendered from the FP32 Gaussians at the
    true pose) reduce the pose error as the FP32 tracker does."""
    from paper_2403_16095_b300 import Rasterizer, Tracker, pack_bf16
    from paper_2403_16095_b300 import _abi as A
    from tests.test_gpu_tracking import _pose_err
    sc = synth.room_scene(80_000, seed=1302)
    cam = synth.Camera(320, 240, 300.0, 300.0, 160.0, 120.0)
    T_gt = synth.room_track_poses(3, seed=1302)[1]
    g32 = to_gpu_gaussians(sc)
    r = Rasterizer([cam], sc.n, tile=16, mode=A.GS_MODE_FWD)
    r.render(g32, poses_gpu(T_gt))
    im = r.frame_images(0)
    tcol, tdep = im["color"].clone(), im["depth"].clone()
    T0 = synth.jitter_pose(T_gt, seed=77, trans=0.02, rot_deg=1.0)
    e0 = _pose_err(T0, T_gt)
    err = {}
    for name, g in (("fp32", g32), ("packed", pack_bf16(g32, spatial=True))):
        tr = Tracker(g, cam, iters=30)
        tr.prepare(tcol, tdep, torch.from_numpy(T0))
        err[name] = _pose_err(tr.track(tcol, tdep, torch.from_numpy(T0)).cpu().numpy(), T_gt)
    print("start (m, deg)", e0, "fp32", err["fp32"], "packed", err["packed"])
    assert err["packed"][0] < 0.8 * e0[0] and err["packed"][1] < 0.6 * e0[1]
    assert err["packed"][0] < err["fp32"][0] + 2e-3
