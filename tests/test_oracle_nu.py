"""Pins of the oracle's per-Gaussian uncertainty estimate (Eq. 13, Sec. 3.2):
dominated pixels (largest blend weight w = alpha T), the weighted squared depth
bias w (D_p - d_i)^2, the mean over all dominated pixels of a keyframe window,
and the tau = 0.025 opacity reset. Expected values come from closed forms of
isotropic Gaussians on the optical axis and from invariants."""
import math

import numpy as np

import oracle
import synth

CAM = synth.Camera(128, 96, 100.0, 100.0, 64.0, 48.0)


def _scene(means, scales, logits, nu=None):
    n = len(means)
    return synth.Scene(np.asarray(means, float), np.log(np.asarray(scales, float))[:, None].repeat(3, 1),
                       np.tile([1.0, 0, 0, 0], (n, 1)), np.asarray(logits, float), np.full((n, 3), 0.5),
                       np.full(n, 0.05) if nu is None else np.asarray(nu, float))


def _pose(tz):
    T = np.zeros((3, 4))
    T[:, :3] = np.eye(3)
    T[2, 3] = tz
    return T


def _alpha_on_axis(s, z, logit):
    """Closed-form alpha of an isotropic Gaussian on the optical axis at depth z
    (Eq. 1-5 with the 0.3 px^2 dilation), the q <= 9 cut and the 1/255 skip."""
    v = (CAM.fx * s / z) ** 2 + 0.3
    xs = np.arange(CAM.width) + 0.5 - CAM.cx
    ys = np.arange(CAM.height) + 0.5 - CAM.cy
    d2 = ys[:, None] ** 2 + xs[None, :] ** 2
    a = np.minimum(0.99, 1.0 / (1.0 + math.exp(-logit)) * np.exp(-d2 / (2 * v)))
    a[d2 / v > 9] = 0
    a[a < 1 / 255] = 0
    return a


def test_single_gaussian_nu_is_mean_weighted_squared_bias_over_window():
    """One Gaussian, two keyframes at different distances: every covered pixel is
    dominated by it (w = alpha), so nu = sum_f sum_p alpha (D_p - z_f)^2 / (M_1 + M_2)."""
    s, z0, logit = 0.06, 2.5, 0.3
    sc = _scene([[0, 0, z0]], [s], [logit])
    rng = np.random.default_rng(1300)
    Ts = [_pose(0.0), _pose(0.7)]
    Ds = [np.full((96, 128), 2.8), rng.uniform(2.0, 4.0, (96, 128))]
    res = oracle.nu_estimate(sc, [CAM, CAM], Ts, Ds)
    num, M = 0.0, 0
    for T, D in zip(Ts, Ds):
        z = z0 + T[2, 3]
        a = _alpha_on_axis(s, z, logit)
        cov = a > 0
        num += float((a[cov] * (D[cov] - z) ** 2).sum())
        M += int(cov.sum())
    assert res["cnt"][0] == M > 100
    np.testing.assert_allclose(res["nu"][0], num / M, rtol=1e-12)
    for f, T in enumerate(Ts):
        a = _alpha_on_axis(s, z0 + T[2, 3], logit)
        assert np.array_equal(res["images"][f]["dominant"], np.where(a > 0, 0, -1))
        np.testing.assert_allclose(res["images"][f]["dom_weight"], a, rtol=0, atol=1e-13)


def test_two_gaussians_dominance_by_hand():
    """A faint front Gaussian over a dense back one on the same axis: w1 = a1,
    w2 = (1 - a1) a2 (Eq. 3-5); each pixel goes to the larger weight (the front
    one on a tie). Near the axis the back Gaussian dominates, in the rim the
    wider front one does."""
    s1, z1, o1 = 0.12, 2.0, -0.85   # sigma ~ 0.30, footprint wider on screen
    s2, z2, o2 = 0.09, 3.5, 2.2     # sigma ~ 0.90
    sc = _scene([[0, 0, z1], [0, 0, z2]], [s1, s2], [o1, o2])
    D = np.full((96, 128), 3.0)
    res = oracle.nu_estimate(sc, [CAM], [_pose(0.0)], [D])
    a1 = _alpha_on_axis(s1, z1, o1)
    a2 = _alpha_on_axis(s2, z2, o2)
    w1, w2 = a1, (1 - a1) * a2
    dom = np.where((w1 == 0) & (w2 == 0), -1, np.where(w1 >= w2, 0, 1))
    assert np.array_equal(res["images"][0]["dominant"], dom)
    assert (dom == 0).sum() > 20 and (dom == 1).sum() > 20
    assert dom[48, 64] == 1
    for i, (w, z) in enumerate(((w1, z1), (w2, z2))):
        m = dom == i
        assert res["cnt"][i] == m.sum()
        np.testing.assert_allclose(res["num"][i], (w[m] * (3.0 - z) ** 2).sum(), rtol=1e-12)
    np.testing.assert_allclose(res["images"][0]["dom_weight"], np.maximum(w1, w2), rtol=0, atol=1e-13)


def test_threshold_lowers_opacity_of_uncertain_gaussians_only():
    """tau = 0.025 (Sec. 3.2): a Gaussian that sits on the sensor depth has nu = 0
    and keeps its opacity; one 0.6 m off it exceeds tau and is lowered to the
    low-opacity level, unless it is already fainter. A Gaussian that dominates
    no pixel keeps its prior nu."""
    sc = _scene([[-0.6, 0, 2.0], [0.6, 0, 2.6], [1.0, 0.8, 5.0], [0, 0, -1.0]], [0.05, 0.05, 0.05, 0.05],
                [1.5, 1.5, -4.8, 0.0], nu=[0.07, 0.0, 0.0, 0.033])
    D = np.full((96, 128), 2.0)
    res = oracle.nu_estimate(sc, [CAM], [_pose(0.0)], [D], tau=0.025, low_opacity=0.01)
    assert res["cnt"][0] > 0 and res["cnt"][1] > 0 and res["cnt"][2] > 0 and res["cnt"][3] == 0
    assert res["nu"][0] == 0.0 and res["nu"][1] > 0.025 and res["nu"][2] > 0.025
    assert res["nu"][3] == 0.033  # behind the camera: culled, nothing dominated
    assert res["over"].tolist() == [False, True, True, True]
    low = math.log(0.01 / 0.99)
    np.testing.assert_allclose(res["opacity_logit"], [1.5, low, -4.8, low], rtol=0, atol=1e-15)


def test_dominated_pixel_invariants_on_random_scene():
    """Every pixel with a blended Gaussian has exactly one dominating Gaussian
    (sum of counts = covered pixels); the dominant weight is the largest of the
    blend weights, so mean weight <= w_max <= accumulated opacity (Eq. 9)."""
    sc, cam, T = synth.tiny_scene()
    tc, td = synth.random_targets(cam, 1301)
    res = oracle.nu_estimate(sc, [cam], [T], [td[0]])
    im = res["images"][0]
    covered = im["n_contrib"] > 0
    assert res["cnt"].sum() == covered.sum() > 5000
    assert np.all((im["dominant"] >= 0) == covered)
    w, O, n = im["dom_weight"][covered], im["alpha"][covered], im["n_contrib"][covered]
    assert np.all(w <= O * (1 + 1e-12)) and np.all(w * n >= O * (1 - 1e-12))
    # a Gaussian's nu is a weighted mean of squared biases: nonnegative, and zero
    # only if every dominated pixel's sensor depth equals its depth
    has = res["cnt"] > 0
    assert np.all(res["nu"][has] > 0)
