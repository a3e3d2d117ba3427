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
from tests.gpu_util import IMG_TOL, at_decision_margin, f32_scene, image_mismatch, poses_gpu, to_gpu_gaussians

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
        bad = image_mismatch(ip, ora, ("color", "depth", "alpha", "nu_map", "T_final"), pix=pix)
        # every differing pixel sits at an FP32/FP64 decision margin; with 5M
        # Gaussians a pixel walks hundreds of entries, so some land near q = 9 or
        # alpha = 1/255: the count is reported (bounded loosely)
        assert np.all(at_decision_margin(ora)[bad]), f"frame {f}: mismatch away from a decision margin"
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


# pixels per frame of the config-5 error report, and its pose-gradient bound
# (max-abs error relative to the largest component); images use IMG_TOL and
# the shared decision margins
PREC_PIX = 8192
PREC_GRAD_TOL = 1e-3


def image_mismatch_err(im, ora, k, pix):
    got = im[k].reshape(3, -1)[:, pix] if k == "color" else im[k].reshape(-1)[pix]
    e = np.abs(got - ora[k])
    return e.max(0) if k == "color" else e


def _gpu_track_grad(r, g, Tg, pix, tc_pix, td_pix, cam):
    """One tracking pass at Tg (forward + POSE backward of the uncertainty-
    weighted L1 loss, lambda = {0.2, 1.0}, tau = 0.025) whose targets equal the
    pass's own colour and depth outside the sampled pixels: their residuals are
    exactly 0 and sign(0) = 0, so only the sampled pixels reach the pose
    gradient. Returns the full-channel images rendered with the sampled sensor
    depth (for U) and the pose gradient."""
    HW = cam.width * cam.height
    r.render(g, Tg)
    zero = torch.zeros(HW, device="cuda")
    r.fwd_bwd_pose(dict(w_color=0.2, w_depth=1.0, unc_tau=0.025, target_color=torch.zeros(3 * HW, device="cuda"),
                        target_depth=zero), images=True)
    col = r.img["color"].clone().view(3, HW)
    dep = r.img["depth"].clone()
    ip = torch.from_numpy(pix).cuda().long()
    col[:, ip] = torch.from_numpy(tc_pix.astype(np.float32)).cuda()
    dep[ip] = torch.from_numpy(td_pix.astype(np.float32)).cuda()
    r.fwd_bwd_pose(dict(w_color=0.2, w_depth=1.0, unc_tau=0.025, target_color=col.reshape(-1), target_depth=dep))
    torch.cuda.synchronize()
    assert r.read_status()[0] == 0
    pg = r.pose_grad[0].cpu().numpy()
    r.render(g, Tg, dep)
    im = {k: v.cpu().numpy() for k, v in r.frame_images(0).items()}
    return im, pg, dep.cpu().numpy()


def test_precision_errors_against_fp64_oracle(precision):
    """Config 5 error report (Eq. 1 storage, Eq. 3-10 outputs, Sec. 3.4 pose
    gradient): on frames 0, 9, 19, ..., 99 of the 1200x680 / 5M workload, at the
    tracker's start pose (2 cm / 1 deg off), 8,192 sampled pixels per frame with
    RGB-D targets from the FP64 oracle at the true pose. For the 16-bit form and
    the FP32 form on the same GPU: colour, depth, opacity and uncertainty U at
    the sampled pixels, and the pose gradient of the tracking loss over them,
    against the FP64 oracle of
      - the decoded 16-bit field (the 16-bit form's arithmetic error),
      - the original field (its total error, storage included),
    and the FP32 form against the oracle of the original field."""
    from paper_2403_16095_b300 import Rasterizer, pack_bf16
    from paper_2403_16095_b300 import _abi as A
    sc, cam, poses = precision
    g32 = to_gpu_gaussians(sc)
    pk = pack_bf16(g32, spatial=True)
    perm = pk.perm.cpu().numpy()
    dec = oracle.unpack_bf16(pk.anchors.cpu().numpy(), pk.packed.cpu().numpy().view(np.uint16))
    orig = f32_scene(sc)
    orig_p = orig.subset(perm)  # the original field in packed order (same index tie-breaks)
    HW = cam.width * cam.height
    rng = np.random.default_rng(1005 + 7)
    rows = []
    worst = {}
    for f in [0] + list(range(9, 100, 10)):
        T_gt = np.asarray(poses[f], np.float32).astype(np.float64)
        T = np.asarray(synth.jitter_pose(poses[f], seed=1005 * 100 + f), np.float32).astype(np.float64)
        pix = np.sort(rng.choice(HW, PREC_PIX, replace=False))
        tgt = oracle.render_pixels(orig, cam, T_gt, pix, mode="rect")
        tc_full = np.zeros((3, HW))
        td_full = np.zeros(HW)
        tc_full[:, pix] = tgt["color"].astype(np.float32)
        td_full[pix] = tgt["depth"].astype(np.float32)
        L = oracle.LossSpec(0.2, 1.0, 0.0, 0.0, 0.025, tc_full.reshape(3, cam.height, cam.width),
                            td_full.reshape(cam.height, cam.width), pixels=pix)
        for form, g, refs in (("16-bit", pk, (("decoded", dec), ("original", orig_p))),
                              ("fp32", g32, (("original", orig),))):
            r = Rasterizer([cam], sc.n, tile=16, mode=A.GS_MODE_POSE)
            im, pg, dep = _gpu_track_grad(r, g, poses_gpu(T), pix, tc_full[:, pix], td_full[pix], cam)
            for ref_name, field in refs:
                ora = oracle.render_pixels(field, cam, T, pix, obs_depth=td_full, mode="rect")
                og = oracle.grad(field, cam, T, L)
                flip = at_decision_margin(ora)
                # reported errors: the sampled pixels away from every decision and
                # depth-order margin (at 5M some frames have none: nan)
                errs = {}
                for k in ("color", "depth", "alpha", "unc"):
                    e = image_mismatch_err(im, ora, k, pix)
                    errs[k] = float(e[~flip].max()) if (~flip).any() else float("nan")
                bad = image_mismatch(im, ora, ("color", "depth", "alpha", "unc"), pix=pix)
                gerr = float(np.abs(pg - og["pose"]).max() / np.abs(og["pose"]).max())
                n_flip = int(bad.sum())
                rows.append((f, form, ref_name, errs, gerr, n_flip))
                key = (form, ref_name)
                w = worst.setdefault(key, dict(color=0.0, depth=0.0, alpha=0.0, unc=0.0, pose=0.0, flips=0))
                for k in errs:
                    w[k] = np.nanmax([w[k], errs[k]])
                w.setdefault("clear_pixels", 0)
                w["clear_pixels"] += int((~flip).sum())
                w["pose"] = max(w["pose"], gerr)
                w["flips"] = max(w["flips"], n_flip)
                if ref_name == "decoded" or form == "fp32":
                    # FP32 arithmetic against FP64 of the same field
                    assert np.all(flip[bad]), (f, form, ref_name, "mismatch away from a margin")
                    assert n_flip <= 0.01 * len(pix), (f, form, ref_name, n_flip)
                    assert gerr < PREC_GRAD_TOL, (f, form, ref_name, gerr)
    for f, form, ref_name, errs, gerr, n_flip in rows:
        print(f"frame {f:3d} {form:6s} vs oracle({ref_name:8s}): " +
              " ".join(f"{k} {v:.2e}" for k, v in errs.items()) + f"  pose-grad rel {gerr:.2e}  "
              f"pixels beyond {IMG_TOL}: {n_flip}")
    for key, w in worst.items():
        print("worst", key, {k: (f"{v:.2e}" if isinstance(v, float) else v) for k, v in w.items()})
