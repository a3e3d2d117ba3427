"""GPU parity of the backward pass (adjoint of Eq. 3-10 through Eq. 1-2, and the
se(3) pose gradient of Sec. 3.4) against the FP64 oracle's analytic gradient,
plus POSE-vs-FULL agreement, determinism, the pose reduction and the Adam step.

Tolerance: gradients are compared per array relative to the array's largest
oracle magnitude. FP32 blending with a reverse walk (T recovered by division,
up to ~100x amplification per entry at alpha = 0.99) over lists of tens of
entries gives ~1e-5 relative error; pixels whose FP32 and FP64 decisions differ
(see the forward test) would perturb single Gaussians more; on these inputs there
are none. Measured on a B300: <= 1.4e-6 of the array's scale per element and
<= 1e-6 for the norm of the difference, so the bounds below (1e-4 per element,
1e-5 for the norm, 1e-5 for the six pose components) leave ~10-70x headroom."""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_util import DECISION_MARGIN, f32_scene, image_mismatch, PARAMS, poses_gpu, to_gpu_gaussians

pytestmark = pytest.mark.gpu


def _setup(mode, sc, cam, T, tile=16):
    from paper_2403_16095_b300 import Rasterizer
    r = Rasterizer([cam], sc.n, tile=tile, mode=mode)
    return r


def _loss_dict(tc, td, w=(1.0, 1.0, 1.0, 1.0, 0.0)):
    return dict(w_color=w[0], w_depth=w[1], w_unc=w[2], w_nu=w[3], unc_tau=w[4],
                w_align=w[5] if len(w) > 5 else 0.0,
                target_color=torch.from_numpy(np.ascontiguousarray(tc)).cuda().reshape(-1),
                target_depth=torch.from_numpy(np.ascontiguousarray(td)).cuda().reshape(-1))


def _spec(w, tc, td):
    return oracle.LossSpec(*w[:5], target_color=tc, target_depth=td, w_align=w[5] if len(w) > 5 else 0.0)


def _run(mode, sc, cam, T, tc, td, w, tile=16):
    from paper_2403_16095_b300 import _abi as A
    g = to_gpu_gaussians(sc)
    Tt = poses_gpu(T)
    r = _setup(mode, sc, cam, T, tile)
    obs = torch.from_numpy(np.ascontiguousarray(td)).cuda().reshape(-1)
    r.render(g, Tt, obs)
    grads = None
    if mode == A.GS_MODE_FULL:
        grads = {k: torch.empty_like(getattr(g, k)) for k in PARAMS}
    r.backward(obs_depth=obs, loss=_loss_dict(tc, td, w), g=g, T_cw=Tt, grads=grads)
    r.reduce_pose()
    torch.cuda.synchronize()
    assert r.read_status()[0] == 0
    return r, grads


def _case(posed=True):
    sc, cam, T = synth.tiny_scene()
    T = np.asarray(T, np.float64)
    if posed:
        c, s = math.cos(0.05), math.sin(0.05)
        T[:, :3] = np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]])
        T[:, 3] = [0.02, -0.04, 0.1]
    tc, td = synth.random_targets(cam, 1001 + 80)
    return sc, cam, np.asarray(T, np.float32).astype(np.float64), tc[0], td[0]


W_ALL = (1.0, 1.0, 1.0, 1.0, 0.0)       # colour + depth + |U| + nu: every parameter gets a gradient
W_TRACK = (0.2, 1.0, 0.0, 0.0, 0.025)   # tracking: lambda = {0.2, 1.0}, uncertainty weighting
W_ALIGN = (0.7, 0.25, 0.0, 0.0, 0.0, 0.25)  # mapping-style weights incl. L_align (Eq. 12, Sec. 4)


def _rel_check(name, got, want, elem=1e-4, norm=1e-5):
    scale = np.abs(want).max()
    assert scale > 0, name
    d = got - want
    e_max = np.abs(d).max() / scale
    e_norm = np.linalg.norm(d) / np.linalg.norm(want)
    print(f"{name}: max {e_max:.2e} norm {e_norm:.2e}")
    assert e_max < elem and e_norm < norm, (name, e_max, e_norm)


@pytest.mark.parametrize("w", [W_ALL, W_TRACK, W_ALIGN])
def test_full_mode_gradients_match_oracle(w):
    from paper_2403_16095_b300 import _abi as A
    sc, cam, T, tc, td = _case()
    r, grads = _run(A.GS_MODE_FULL, sc, cam, T, tc, td, w)
    L = _spec(w, tc, td)
    og = oracle.grad(f32_scene(sc), cam, T, L)
    for k in PARAMS:
        if k == "nu" and w[3] == 0:
            assert float(grads[k].abs().max()) == 0.0
            continue
        _rel_check(k, grads[k].cpu().numpy().astype(np.float64), og[k])
    _rel_check("pose", r.pose_grad[0].cpu().numpy(), og["pose"], elem=1e-5, norm=1e-5)


def test_full_mode_repeated_calls_on_one_workspace():
    """Three FULL backward calls on one Rasterizer (one workspace), two of
    them with a forward between, give the same gradients, up to the arrival
    order of the per-record accumulators' atomics, and match the oracle: no
    call sees another's accumulators, and the projection adjoint's
    visibility (tiles_touched) is the projection's."""
    from paper_2403_16095_b300 import _abi as A
    sc, cam, T, tc, td = _case()
    g = to_gpu_gaussians(sc)
    Tt = poses_gpu(T)
    r = _setup(A.GS_MODE_FULL, sc, cam, T, 16)
    obs = torch.from_numpy(np.ascontiguousarray(td)).cuda().reshape(-1)
    runs = []
    for k in range(3):
        if k != 1:  # the second call reuses the first call's forward
            r.render(g, Tt, obs)
        grads = {p: torch.empty_like(getattr(g, p)) for p in PARAMS}
        r.backward(obs_depth=obs, loss=_loss_dict(tc, td, W_ALL), g=g, T_cw=Tt, grads=grads)
        torch.cuda.synchronize()
        assert r.read_status()[0] == 0
        runs.append({p: v.cpu().numpy().astype(np.float64) for p, v in grads.items()})
    og = oracle.grad(f32_scene(sc), cam, T, _spec(W_ALL, tc, td))
    for p in PARAMS:
        scale = np.abs(runs[0][p]).max()
        for k in (1, 2):
            assert np.abs(runs[k][p] - runs[0][p]).max() <= 1e-5 * scale, (p, k)
        _rel_check(p, runs[2][p], og[p])


def test_pose_mode_matches_full_mode_and_oracle():
    """P10c: the per-pixel Jacobian contraction (POSE) and the per-Gaussian
    reverse chain (FULL) give the same pose gradient."""
    from paper_2403_16095_b300 import _abi as A
    sc, cam, T, tc, td = _case()
    rp, _ = _run(A.GS_MODE_POSE, sc, cam, T, tc, td, W_TRACK)
    rf, _ = _run(A.GS_MODE_FULL, sc, cam, T, tc, td, W_TRACK)
    gp = rp.pose_grad[0].cpu().numpy()
    gf = rf.pose_grad[0].cpu().numpy()
    np.testing.assert_allclose(gp, gf, rtol=0, atol=2e-5 * np.abs(gf).max())
    og = oracle.grad(f32_scene(sc), cam, T, oracle.LossSpec(*W_TRACK, target_color=tc, target_depth=td))
    _rel_check("pose(POSE mode)", gp, og["pose"], elem=1e-5, norm=1e-5)


@pytest.mark.parametrize("tile", [8, 32])
def test_pose_mode_other_tile_sizes(tile):
    from paper_2403_16095_b300 import _abi as A
    sc, cam, T, tc, td = _case()
    r16, _ = _run(A.GS_MODE_POSE, sc, cam, T, tc, td, W_TRACK, tile=16)
    rt, _ = _run(A.GS_MODE_POSE, sc, cam, T, tc, td, W_TRACK, tile=tile)
    a, b = r16.pose_grad[0].cpu().numpy(), rt.pose_grad[0].cpu().numpy()
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-5 * np.abs(a).max())


def test_pose_gradient_bit_identical_across_runs():
    """P12: fixed reduction trees, no atomics in POSE mode."""
    from paper_2403_16095_b300 import _abi as A
    sc, cam, T, tc, td = _case()
    a, _ = _run(A.GS_MODE_POSE, sc, cam, T, tc, td, W_TRACK)
    b, _ = _run(A.GS_MODE_POSE, sc, cam, T, tc, td, W_TRACK)
    assert torch.equal(a.pose_grad, b.pose_grad)
    assert torch.equal(a.pose_partials, b.pose_partials)


def test_fused_loss_equals_upstream_gradient_maps():
    """The fused loss inside the backward kernel and the same per-pixel gradient
    supplied as dL maps give the same pose gradient."""
    from paper_2403_16095_b300 import _abi as A
    sc, cam, T, tc, td = _case()
    r, _ = _run(A.GS_MODE_POSE, sc, cam, T, tc, td, (1.0, 1.0, 0.0, 0.0, 0.0))
    fused = r.pose_grad.clone()
    im = r.frame_images(0)
    HW = cam.width * cam.height
    tct = torch.from_numpy(tc).cuda()
    tdt = torch.from_numpy(td).cuda()
    dL = {"color": (torch.sign(im["color"] - tct) / HW).contiguous().reshape(-1),
          "depth": (torch.sign(im["depth"] - tdt) / HW).contiguous().reshape(-1)}
    obs = tdt.reshape(-1)
    r.backward(obs_depth=obs, dL=dL)
    r.reduce_pose()
    torch.cuda.synchronize()
    np.testing.assert_allclose(r.pose_grad.cpu().numpy(), fused.cpu().numpy(), rtol=1e-6, atol=1e-9)


def test_autograd_function_matches_oracle():
    """torch.autograd through GaussianRasterize (FULL backward with upstream maps
    from a torch loss) vs the oracle's analytic gradient of the same loss."""
    from paper_2403_16095_b300 import Rasterizer, rasterize
    from paper_2403_16095_b300 import _abi as A
    sc, cam, T, tc, td = _case()
    g = to_gpu_gaussians(sc)
    for k in PARAMS:
        getattr(g, k).requires_grad_(True)
    xi = torch.zeros(1, 6, device="cuda", requires_grad=True)
    r = Rasterizer([cam], sc.n, tile=16, mode=A.GS_MODE_FULL)
    obs = torch.from_numpy(td).cuda().reshape(-1)
    out = rasterize(g, xi, poses_gpu(T), r, obs)
    HW = cam.width * cam.height
    loss = ((out["color"] - torch.from_numpy(tc).cuda().reshape(-1)).abs().sum()
            + (out["depth"] - obs).abs().sum() + out["unc"].abs().sum() + out["nu_map"].sum()) / HW
    loss.backward()
    og = oracle.grad(f32_scene(sc), cam, T, oracle.LossSpec(*W_ALL, target_color=tc, target_depth=td))
    assert abs(float(loss.detach()) - og["loss"]) < 1e-4 * og["loss"]
    for k in PARAMS:
        _rel_check(k, getattr(g, k).grad.cpu().numpy().astype(np.float64), og[k])
    _rel_check("xi", xi.grad[0].cpu().numpy().astype(np.float64), og["pose"], elem=1e-5, norm=1e-5)


def test_pose_grad_reduce_is_exactly_rounded_sum():
    from paper_2403_16095_b300 import _abi as A
    rng = np.random.default_rng(0)
    F, K = 3, 1777
    vals = rng.normal(size=(F, K, 6)) * np.exp(rng.uniform(-20, 20, size=(F, K, 6)))
    hi = vals.astype(np.float32)
    lo = (vals - hi.astype(np.float64)).astype(np.float32)
    parts = hi.astype(np.float64) + lo.astype(np.float64)  # the exact values passed in
    pt = torch.from_numpy(np.stack([hi, lo], -1).reshape(-1)).cuda()
    out = torch.zeros(F, 6, dtype=torch.float64, device="cuda")
    st = torch.zeros(4, dtype=torch.int32, device="cuda")
    A.gs_pose_grad_reduce(pt, F, K, out, st)
    torch.cuda.synchronize()
    want = np.array([[math.fsum(parts[f, :, k]) for k in range(6)] for f in range(F)])
    got = out.cpu().numpy()
    # double-float sums carry ~48 bits: error below 1e-12 of the summed magnitudes
    assert np.all(np.abs(got - want) <= 1e-12 * np.abs(parts).sum(1))


def test_fused_pose_reduction_equals_standalone_call():
    """The last-CTA reduction inside gs_render_bwd and gs_pose_grad_reduce run the
    same fixed-order sum: bit-identical, in POSE and FULL mode."""
    from paper_2403_16095_b300 import _abi as A
    sc, cam, T, tc, td = _case()
    for mode in (A.GS_MODE_POSE, A.GS_MODE_FULL):
        r, _ = _run(mode, sc, cam, T, tc, td, W_TRACK)  # backward writes the fused pose_grad
        fused = r.pose_grad.clone()
        r.pose_grad.zero_()
        r.reduce_pose()
        torch.cuda.synchronize()
        assert torch.equal(fused, r.pose_grad), mode


def test_adam_step_matches_oracle():
    from paper_2403_16095_b300 import _abi as A
    from paper_2403_16095_b300.raster import pose_state
    rng = np.random.default_rng(1)
    T = np.c_[np.eye(3), [0.3, -1.2, 2.0]]
    st_o = np.zeros(25)
    st_o[:9] = np.eye(3).reshape(-1)
    st_o[9:12] = T[:, 3]
    st_g = pose_state(torch.from_numpy(T).cuda())
    Tf = torch.zeros(12, device="cuda")
    status = torch.zeros(4, dtype=torch.int32, device="cuda")
    adam = A.gs_adam(0.0015, 0.00215, 0.9, 0.999, 1e-8)
    f32 = [float(np.float32(v)) for v in (0.0015, 0.00215, 0.9, 0.999, 1e-8)]  # the ABI passes FP32
    for _ in range(5):
        gr = rng.normal(size=6)
        oracle.adam_step(st_o, gr, *f32)
        A.gs_pose_adam_step(st_g, torch.from_numpy(gr).cuda(), Tf, 1, adam, status)
    torch.cuda.synchronize()
    got = st_g[0].cpu().numpy()
    # moments and step count: the same FP64 recurrences; the rotation moments see
    # t through g_R = g_phi - t x g_rho, so they inherit the FP32-step difference
    np.testing.assert_allclose(got[12:25], st_o[12:25], rtol=1e-8, atol=1e-15)
    # the step d is evaluated in FP32 (|d| <= ~3 lr): pose within 1e-6 of each step
    np.testing.assert_allclose(got[:12], st_o[:12], rtol=0, atol=5 * 1e-6 * 0.00215)
    np.testing.assert_allclose(got[25:27], [float(np.float32(0.9)) ** 5, float(np.float32(0.999)) ** 5], rtol=1e-14)
    want = np.c_[st_o[:9].reshape(3, 3), st_o[9:12]].reshape(-1)
    np.testing.assert_allclose(Tf.cpu().numpy(), want, rtol=0, atol=1e-6)


def _degenerate_scene():
    """tiny_scene with the degenerate Gaussians the method meets: zero
    quaternions (invalid: culled, zero gradient), saturated opacity (alpha
    clamped at 0.99, so no opacity gradient through the clamp), sub-pixel
    scales (footprint from the 0.3 px^2 dilation alone), one Gaussian covering
    every tile, centres outside the image whose footprints reach in (ten at one
    depth: ties ordered by index), and means just in front of and behind the
    near plane."""
    sc, cam, T = synth.tiny_scene(n=800, seed=1401)
    m, ls, q, o = sc.means.copy(), sc.log_scales.copy(), sc.quats.copy(), sc.opacity_logit.copy()
    q[0:20] = 0.0
    o[20:30] = 20.0
    ls[30:40] = -9.0
    m[40], ls[40], o[40] = (0.0, 0.0, 3.0), np.log(2.0), -1.0
    for k, i in enumerate(range(41, 51)):
        side = 1.0 if k % 2 else -1.0
        m[i] = (side * 1.48, 0.3 * (k / 10.0 - 0.5), 2.0) if k < 6 else (0.2 * k - 1.4, side * 1.1, 2.0)
        ls[i] = np.log(0.1)
    m[51:53, 2] = 0.19   # behind the near plane (0.2): culled
    m[53:56, 2] = 0.21   # just in front of it: large footprints
    m[53:56, :2] = [[0.0, 0.0], [0.01, -0.01], [-0.02, 0.015]]
    f = np.float32
    sc2 = synth.Scene(m.astype(f), ls.astype(f), q.astype(f), o.astype(f), sc.colors, sc.nu)
    return sc2, cam, T


def test_degenerate_gaussians_match_oracle():
    from paper_2403_16095_b300 import _abi as A
    sc, cam, T = _degenerate_scene()
    T = np.asarray(T, np.float32).astype(np.float64)
    tc, td = synth.random_targets(cam, 1401 + 1)
    r, grads = _run(A.GS_MODE_FULL, sc, cam, T, tc[0], td[0], W_ALL)
    ora = oracle.render(f32_scene(sc), cam, T, obs_depth=td[0])
    im = {k: v.cpu().numpy() for k, v in r.frame_images(0).items()}
    bad = image_mismatch(im, ora, ("color", "depth", "alpha", "unc", "nu_map", "T_final"))
    # a differing pixel must sit at an FP32-vs-FP64 decision flip (the depth-gap
    # margin, channel 4, is left out: equal depths are ordered by index on both
    # sides, and the ten Gaussians outside the image share z = 2)
    flip = ora["margins"][[0, 1, 2, 3, 5]].min(axis=0)
    assert np.all(flip[bad] < DECISION_MARGIN) and int(bad.sum()) <= 3, int(bad.sum())
    og = oracle.grad(f32_scene(sc), cam, T, _spec(W_ALL, tc[0], td[0]))
    for k in PARAMS:
        got = grads[k].cpu().numpy()
        assert np.all(got[0:20] == 0.0) and np.all(got[51:53] == 0.0), k  # culled: exactly zero
        assert np.all(og[k][0:20] == 0.0) and np.all(og[k][51:53] == 0.0), k
        _rel_check(k, got.astype(np.float64), og[k])
    _rel_check("pose", r.pose_grad[0].cpu().numpy(), og["pose"], elem=1e-5, norm=1e-5)
    # the degenerate Gaussians do reach the image: the covering one and the
    # near-plane ones get gradients
    assert np.abs(og["means"][40]).max() > 0 and np.abs(og["means"][53:56]).max() > 0
    rp, _ = _run(A.GS_MODE_POSE, sc, cam, T, tc[0], td[0], W_ALL)
    _rel_check("pose(POSE mode)", rp.pose_grad[0].cpu().numpy(), og["pose"], elem=1e-5, norm=1e-5)
