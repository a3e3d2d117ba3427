"""Pins of the oracle's sampled and windowed evaluations.

* Central differences of a keyframe window's loss (Eq. 21), re-blending only
  the pixels the perturbed Gaussian can reach (``oracle.fd_window``), against
  (a) differences of full-image loss sums and (b) the analytic adjoint summed
  over the window's frames.
* The pixel subset of the loss (``LossSpec.pixels``) and the row-list sampled
  render against their full-image counterparts: a loss over a subset plus the
  loss over its complement is the full loss (value and gradient), and a
  sampled pixel renders exactly as in the full image.
"""
import math

import numpy as np

import oracle
import synth


def _posed(T, xi):
    rho, phi = np.asarray(xi[:3], float), np.asarray(xi[3:], float)
    th = np.linalg.norm(phi)
    K = np.array([[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]])
    R = np.eye(3) if th == 0 else np.eye(3) + math.sin(th) / th * K + (1 - math.cos(th)) / th ** 2 * K @ K
    out = np.zeros((3, 4))
    out[:, :3] = R @ T[:, :3]
    out[:, 3] = R @ T[:, 3] + rho
    return out


def _full_loss(sc, cam, T, L):
    return oracle.loss_value(sc, cam, T, L)


def _set(sc, k, i, v):
    """Parameter k (FD_PARAMS order) of Gaussian i."""
    off = 0
    for name, dim in oracle.FD_PARAMS:
        if k < off + dim:
            arr = getattr(sc, name)
            if arr.ndim == 2:
                old = arr[i, k - off]
                arr[i, k - off] = v(old)
            else:
                old = arr[i]
                arr[i] = v(old)
            return old
        off += dim


def test_fd_window_equals_full_image_differences():
    """O14: per element, the windowed difference equals the difference of two
    full-image loss sums (every pixel blended) wherever neither evaluation
    changes a decision; an element the window marks stable is also stable for
    the full image."""
    sc, cam, T = synth.fd_scene()
    tc, td = synth.random_targets(cam, 1100 + 31, depth_range=(2, 4))
    L = oracle.LossSpec(0.7, 0.25, 0.15, 0.1, 0.0, tc[0], td[0], w_align=0.25)
    h = 1e-4
    sel = np.arange(sc.n)
    fd, st = oracle.fd_window(sc, [cam], [T], [L], sel, h=h)
    _, h0 = _full_loss(sc, cam, T, L)
    n_cmp = 0
    for s, i in enumerate(sel):
        for k in range(15):
            _set(sc, k, i, lambda o: o + h)
            vp, hp = _full_loss(sc, cam, T, L)
            _set(sc, k, i, lambda o: o - 2 * h)
            vm, hm = _full_loss(sc, cam, T, L)
            _set(sc, k, i, lambda o: o + h)
            full_stable = hp == h0 and hm == h0
            if st[s, k]:
                assert full_stable, (i, k)
                want = (vp - vm) / (2 * h)
                # the full-image sums round at ~1e-16 of the loss (~1): 1e-11 after / 2h
                assert abs(fd[s, k] - want) <= 1e-9 * abs(want) + 1e-11, (i, k, fd[s, k], want)
                n_cmp += 1
    assert n_cmp >= 0.8 * 15 * sc.n


def test_fd_window_matches_analytic_gradient_over_frames():
    """O14 against O12: over a three-frame window with every loss term of the
    rasterizer path (colour, depth, |U|, nu map, L_align), the windowed central
    differences equal the analytic FP64 gradients summed over the frames to
    1e-6 relative on the elements whose active set is stable."""
    sc, cam, T = synth.fd_scene()
    Ts = [T, _posed(T, [0.03, -0.02, 0.05, 0.02, -0.01, 0.03]), _posed(T, [-0.04, 0.01, -0.03, -0.02, 0.03, 0.0])]
    Ls = []
    for f in range(3):
        tc, td = synth.random_targets(cam, 1100 + 40 + f, depth_range=(2, 4))
        Ls.append(oracle.LossSpec(0.7, 0.25, 0.15, 0.1, 0.0, tc[0], td[0], w_align=0.25))
    sel = np.arange(sc.n)
    fd, st = oracle.fd_window(sc, [cam] * 3, Ts, Ls, sel, h=1e-4)
    ana = np.zeros((sc.n, 15))
    for T_f, L_f in zip(Ts, Ls):
        g = oracle.grad(sc, cam, T_f, L_f)
        ana += np.concatenate([g[name].reshape(sc.n, -1) for name, _ in oracle.FD_PARAMS], 1)
    scale = np.abs(ana).max(0)
    err = np.abs(fd - ana) / np.maximum(scale, 1e-12)
    assert st.mean() > 0.7
    assert err[st].max() < 1e-6, err[st].max()


def test_pixel_subset_loss_and_gradient_add_up_to_the_full_image():
    """A loss over a pixel subset plus the loss over its complement is the full
    loss, for the value and for every gradient (the sum is linear in pixels);
    the subset keeps the image's 1/(HW) factor."""
    sc, cam, T = synth.fd_scene()
    tc, td = synth.random_targets(cam, 1100 + 51, depth_range=(2, 4))
    HW = cam.width * cam.height
    rng = np.random.default_rng(3)
    sub = np.sort(rng.choice(HW, HW // 3, replace=False))
    comp = np.setdiff1d(np.arange(HW), sub)
    mk = lambda pix: oracle.LossSpec(0.2, 1.0, 0.15, 0.1, 0.025, tc[0], td[0], w_align=0.25, pixels=pix)
    full = oracle.grad(sc, cam, T, mk(None))
    a = oracle.grad(sc, cam, T, mk(sub))
    b = oracle.grad(sc, cam, T, mk(comp))
    assert abs(a["loss"] + b["loss"] - full["loss"]) <= 1e-14 * full["loss"]
    assert 0 < a["loss"] < full["loss"]
    for k in ("means", "log_scales", "quats", "opacity_logit", "colors", "nu", "pose"):
        np.testing.assert_allclose(a[k] + b[k], full[k], rtol=0, atol=1e-12 * np.abs(full[k]).max())
    va, _ = oracle.loss_value(sc, cam, T, mk(sub))
    assert abs(va - a["loss"]) <= 1e-14 * va


def test_sampled_render_row_lists_equal_full_image():
    """A sampled pixel rendered from the row lists, and by brute force, equals
    the same pixel of the full render bit for bit (same list, same order)."""
    sc, cam, T = synth.tiny_scene()
    _, td = synth.random_targets(cam, 1001 + 52)
    full = oracle.render(sc, cam, T, obs_depth=td[0])
    HW = cam.width * cam.height
    pix = np.random.default_rng(4).choice(HW, 500, replace=False)
    for mode in ("rect", "brute"):
        s = oracle.render_pixels(sc, cam, T, pix, obs_depth=td[0], mode=mode)
        for k in ("depth", "alpha", "unc", "nu_map", "median", "T_final", "n_contrib"):
            assert np.array_equal(s[k], full[k].reshape(-1)[pix]), (mode, k)
        assert np.array_equal(s["color"], full["color"].reshape(3, -1)[:, pix]), mode
