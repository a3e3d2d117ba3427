"""Pins of the FP64 CPU oracle against facts fixed by the paper's definitions and
by mathematics (closed forms, invariants, brute force, finite differences).

Each test names the equation it pins. None of these compares the oracle with
itself through a retyped formula: every expected value comes from an
independent route (a closed form for a special case, an invariant, a second
algorithm, or numerical differentiation).
"""

import math

import numpy as np
import pytest

import oracle
import synth


def _scene(means, log_scales, quats, logits, colors, nu=None):
    n = len(means)
    return synth.Scene(np.asarray(means, float), np.asarray(log_scales, float), np.asarray(quats, float),
                       np.asarray(logits, float), np.asarray(colors, float),
                       np.zeros(n) if nu is None else np.asarray(nu, float))


def _ident():
    T = np.zeros((3, 4))
    T[:, :3] = np.eye(3)
    return T


CAM = synth.Camera(128, 96, 100.0, 100.0, 64.0, 48.0)


# ----------------------------------------------------------- Eq. 1-5 closed form
def test_single_isotropic_gaussian_closed_form():
    """P1 (Eq. 1-5 with the 0.3 px^2 dilation): one isotropic Gaussian at (0,0,z)
    renders alpha(p) = sigma exp(-|d|^2 / (2 v)), v = (f s / z)^2 + 0.3, inside
    q <= 9, and its footprint radius is ceil(3 sqrt(v))."""
    z, s, logit = 3.0, 0.05, 0.4
    sc = _scene([[0, 0, z]], [[math.log(s)] * 3], [[0.3, -0.5, 0.7, 0.1]], [logit], [[1.0, 0.5, 0.25]])
    im = oracle.render(sc, CAM, _ident())
    pr = oracle.project(sc, CAM, _ident())
    v = (CAM.fx * s / z) ** 2 + 0.3
    sigma = 1.0 / (1.0 + math.exp(-logit))
    assert pr["radius"][0] == math.ceil(3 * math.sqrt(v))
    np.testing.assert_allclose(pr["mean2d"][0], [64.0, 48.0], rtol=0, atol=1e-12)
    np.testing.assert_allclose(pr["conic"][0], [1 / v, 0, 1 / v], rtol=1e-12, atol=1e-15)
    xs = np.arange(128) + 0.5 - 64.0
    ys = np.arange(96) + 0.5 - 48.0
    d2 = ys[:, None] ** 2 + xs[None, :] ** 2
    alpha = sigma * np.exp(-d2 / (2 * v))
    alpha[d2 / v > 9] = 0
    alpha[alpha < 1 / 255] = 0
    np.testing.assert_allclose(im["alpha"], alpha, rtol=0, atol=1e-12)
    np.testing.assert_allclose(im["color"][1], 0.5 * alpha, rtol=0, atol=1e-12)
    np.testing.assert_allclose(im["depth"], z * alpha, rtol=0, atol=1e-12)


def test_principal_point_symmetry():
    """P2 (pixel-centre convention): with cx = W/2, cy = H/2 the image of an
    isotropic Gaussian on the optical axis is mirror-symmetric, bit for bit."""
    sc = _scene([[0, 0, 2.5]], [[math.log(0.04)] * 3], [[1, 0, 0, 0]], [1.0], [[0.2, 0.9, 0.4]])
    im = oracle.render(sc, CAM, _ident())
    a = im["alpha"]
    assert np.array_equal(a, a[:, ::-1]) and np.array_equal(a, a[::-1, :])
    assert a[47, 63] == a[48, 64] > 0.5


# ----------------------------------------------------------- Eq. 6-10 wiring
def test_fronto_parallel_opaque_depth_and_uncertainty():
    """P3 (Eq. 6-10): a stack of flat, opaque Gaussians all at depth z gives
    D_alpha / O = z, median depth z, and U = 0 when the sensor depth is z."""
    z = 2.0
    rng = np.random.default_rng(3)
    n = 12
    means = np.c_[rng.uniform(-0.1, 0.1, n), rng.uniform(-0.1, 0.1, n), np.full(n, z)]
    ls = np.c_[np.full(n, math.log(0.08)), np.full(n, math.log(0.08)), np.full(n, math.log(1e-4))]
    sc = _scene(means, ls, np.tile([1.0, 0, 0, 0], (n, 1)), np.full(n, 6.0), rng.uniform(0, 1, (n, 3)))
    D = np.full((96, 128), z)
    im = oracle.render(sc, CAM, _ident(), obs_depth=D)
    cov = im["alpha"] > 0.5
    assert cov.sum() > 200
    np.testing.assert_allclose(im["depth"][cov] / im["alpha"][cov], z, rtol=1e-14)
    assert np.all(im["median"][cov] == z)
    assert np.all(im["unc"] == 0.0)
    # an opaque single Gaussian saturates at the 0.99 clamp in its centre
    one = oracle.render(sc.subset([0]), CAM, _ident())
    assert abs(one["alpha"].max() - 0.99) < 1e-12


def test_median_depth_is_first_crossing_of_half():
    """Eq. 7-8: the median depth is the depth of the Gaussian at which T first
    drops below 0.5; with alphas 0.3 then 0.4 (T: 1 -> 0.7 -> 0.42) it is the
    second one."""
    # two Gaussians straddling the centre pixel; alpha at the centre pixel set via opacity
    v = (100 * 0.05 / 2.0) ** 2 + 0.3
    g = math.exp(-0.5 * 0.5 / v)                     # centre pixel offset (0.5, 0.5)
    lo1 = -math.log(1.0 / (0.3 / g) - 1)             # alpha_1 = 0.3 at that pixel
    g2 = math.exp(-0.5 * 0.5 / ((100 * 0.05 / 3.0) ** 2 + 0.3))
    lo2 = -math.log(1.0 / (0.4 / g2) - 1)
    sc = _scene([[0, 0, 2.0], [0, 0, 3.0]], [[math.log(0.05)] * 3] * 2, [[1, 0, 0, 0]] * 2, [lo1, lo2],
                [[1, 0, 0], [0, 1, 0]])
    im = oracle.render(sc, CAM, _ident())
    assert im["median"][48, 64] == 3.0
    np.testing.assert_allclose(im["T_final"][48, 64], 0.7 * 0.6, rtol=1e-12)


def test_two_gaussian_composite_by_hand():
    """P5 (Eq. 3-4): front Gaussian 1, back Gaussian 2 on the same ray:
    C = a1 c1 + (1 - a1) a2 c2 at every pixel both cover."""
    s1, z1, o1, s2, z2, o2 = 0.06, 2.0, 0.2, 0.09, 3.5, 1.1
    c1, c2 = np.array([0.9, 0.1, 0.3]), np.array([0.2, 0.8, 0.5])
    sc = _scene([[0.0, 0, z1], [0.0, 0, z2]], [[math.log(s1)] * 3, [math.log(s2)] * 3],
                [[1, 0, 0, 0], [0, 0, 1, 0]], [o1, o2], [c1, c2])
    im = oracle.render(sc, CAM, _ident())
    for (px, py) in [(64, 48), (66, 47), (60, 50)]:
        d2 = (px + 0.5 - 64) ** 2 + (py + 0.5 - 48) ** 2
        a1 = 1 / (1 + math.exp(-o1)) * math.exp(-d2 / (2 * ((100 * s1 / z1) ** 2 + 0.3)))
        a2 = 1 / (1 + math.exp(-o2)) * math.exp(-d2 / (2 * ((100 * s2 / z2) ** 2 + 0.3)))
        want = a1 * c1 + (1 - a1) * a2 * c2
        np.testing.assert_allclose(im["color"][:, py, px], want, rtol=1e-12)
        np.testing.assert_allclose(im["depth"][py, px], a1 * z1 + (1 - a1) * a2 * z2, rtol=1e-12)


def test_projection_of_rotated_anisotropic_gaussian():
    """Eq. 1-2 at the image centre: for a point on the optical axis J W = (f/z) [I2 | 0]
    (identity pose), so Sigma_2d = (f/z)^2 [R S^2 R^T]_{2x2} + 0.3 I and the conic is
    its inverse; checked with an explicit axis-angle rotation (not a quaternion)."""
    ang, z, f = 0.6, 2.0, 100.0
    s = np.array([0.02, 0.07, 0.01])
    # quaternion of a rotation by ang about z
    q = [math.cos(ang / 2), 0, 0, math.sin(ang / 2)]
    sc = _scene([[0, 0, z]], [np.log(s)], [q], [0.0], [[1, 1, 1]])
    pr = oracle.project(sc, CAM, _ident())
    c, sn = math.cos(ang), math.sin(ang)
    R2 = np.array([[c, -sn], [sn, c]])
    cov = (f / z) ** 2 * R2 @ np.diag(s[:2] ** 2) @ R2.T + 0.3 * np.eye(2)
    inv = np.linalg.inv(cov)
    np.testing.assert_allclose(pr["conic"][0], [inv[0, 0], inv[0, 1], inv[1, 1]], rtol=1e-12)


def test_footprint_ellipse_lies_inside_the_pixel_rect():
    """Footprint (Eq. 2 radius and rect): every pixel with q <= 9 lies in the
    Gaussian's pixel rect, so a pixel's list is decided by q alone within the
    tiles the rect covers. Checked by brute force over a margin of 3 pixels
    around every rect, on anisotropic, rotated Gaussians, including ones whose
    projection Jacobian is clamped at the image edge; q is evaluated both in
    FP64 and in FP32 from the FP32-rounded centre and conic, as the kernels
    do."""
    scenes = [synth.tiny_scene(n=400, seed=1401)[0], synth.fd_scene(n=60, seed=1402, n_edge=8)[0]]
    cams = [synth.Camera(128, 96, 100.0, 100.0, 64.0, 48.0), synth.Camera(64, 48, 60.0, 60.0, 32.0, 24.0)]
    checked = 0
    for sc, cam in zip(scenes, cams):
        pr = oracle.project(sc, cam, _ident())
        for g in np.flatnonzero(pr["valid"]):
            x0, y0, x1, y1 = pr["rect"][g]
            mx, my = pr["mean2d"][g]
            A, B, C = pr["conic"][g]
            xs = np.arange(max(0, x0 - 3), min(cam.width, x1 + 4))
            ys = np.arange(max(0, y0 - 3), min(cam.height, y1 + 4))
            px, py = np.meshgrid(xs, ys)
            inside = (px >= x0) & (px <= x1) & (py >= y0) & (py <= y1)
            dx, dy = px + 0.5 - mx, py + 0.5 - my
            q64 = A * dx * dx + 2 * B * dx * dy + C * dy * dy
            f = np.float32
            dx32, dy32 = f(px + 0.5) - f(mx), f(py + 0.5) - f(my)
            q32 = f(A) * dx32 * dx32 + f(2) * f(B) * dx32 * dy32 + f(C) * dy32 * dy32
            assert not np.any((q64 <= 9.0) & ~inside), g
            assert not np.any((q32 <= f(9.0)) & ~inside), g
            checked += int(np.count_nonzero(q64 <= 9.0))
    assert checked > 10_000


# ----------------------------------------------------------- invariants (P4)
@pytest.fixture(scope="module")
def tiny():
    sc, cam, T = synth.tiny_scene()
    _, td = synth.random_targets(cam, 1001 + 50)
    im = oracle.render(sc, cam, T, obs_depth=td[0])
    return sc, cam, T, im


def test_blend_invariants(tiny):
    """P4 (Eq. 3-10): O in [0, 1 - 1e-4]; O = 1 - T_final; C <= max(c) O;
    D_alpha within [zmin O, zmax O]; U >= 0; nu map within [0, max nu * O]."""
    sc, cam, T, im = tiny
    O = im["alpha"]
    assert O.min() >= 0 and O.max() <= 1 - 1e-4 + 1e-15
    np.testing.assert_allclose(O, 1 - im["T_final"], rtol=0, atol=1e-12)
    cmax = sc.colors.max(0)
    for c in range(3):
        assert np.all(im["color"][c] <= cmax[c] * O + 1e-12)
    z = sc.means[:, 2].astype(float)
    assert np.all(im["depth"] <= z.max() * O + 1e-12) and np.all(im["depth"] >= z.min() * O - 1e-12)
    assert im["unc"].min() >= 0
    assert np.all(im["nu_map"] <= sc.nu.max() * O + 1e-12)
    assert im["n_contrib"].max() > 20


def test_uniform_color_equals_color_times_opacity(tiny):
    """Eq. 3 and 9: with every Gaussian coloured c the image is c * O."""
    sc, cam, T, _ = tiny
    sc2 = synth.Scene(sc.means, sc.log_scales, sc.quats, sc.opacity_logit,
                      np.tile(np.array([0.25, 0.5, 0.75], np.float32), (sc.n, 1)), sc.nu)
    im = oracle.render(sc2, cam, T)
    for c, v in enumerate([0.25, 0.5, 0.75]):
        np.testing.assert_allclose(im["color"][c], v * im["alpha"], rtol=1e-13, atol=1e-15)


def test_brute_force_equals_rect_scatter(tiny):
    """P6: per-pixel brute force over all Gaussians and the rect-scatter lists give
    bit-identical FP64 images."""
    sc, cam, T, im = tiny
    _, td = synth.random_targets(cam, 1001 + 50)
    im2 = oracle.render(sc, cam, T, obs_depth=td[0], mode="brute")
    for k in im:
        assert np.array_equal(im[k], im2[k]), k


def test_sampled_pixels_equal_full_image(tiny):
    sc, cam, T, im = tiny
    _, td = synth.random_targets(cam, 1001 + 50)
    pix = np.random.default_rng(0).choice(cam.width * cam.height, 300, replace=False)
    s = oracle.render_pixels(sc, cam, T, pix, obs_depth=td[0])
    for k in ("depth", "alpha", "unc", "nu_map", "median", "T_final"):
        assert np.array_equal(s[k], im[k].reshape(-1)[pix]), k
    assert np.array_equal(s["color"], im["color"].reshape(3, -1)[:, pix])


def test_stop_rule_never_lets_T_below_1e4():
    """The blend stops before an entry that would take T below 1e-4: a deep stack
    of nearly opaque Gaussians on the optical axis keeps two entries at the
    centre pixel, T_final = (1-a1)(1-a2) >= 1e-4 while (1-a3) T_final < 1e-4."""
    n, s, sig = 30, 0.2, 0.97
    z = np.linspace(2, 3, n)
    sc = _scene(np.c_[np.zeros(n), np.zeros(n), z], np.full((n, 3), math.log(s)),
                np.tile([1.0, 0, 0, 0], (n, 1)), np.full(n, math.log(sig / (1 - sig))), np.full((n, 3), 0.5))
    im = oracle.render(sc, CAM, _ident())
    assert im["T_final"].min() >= 1e-4
    a = [sig * math.exp(-0.25 / ((100 * s / zk) ** 2 + 0.3)) for zk in z[:3]]
    assert im["n_contrib"][48, 64] == 2
    np.testing.assert_allclose(im["T_final"][48, 64], (1 - a[0]) * (1 - a[1]), rtol=1e-12)
    assert (1 - a[2]) * im["T_final"][48, 64] < 1e-4


# ----------------------------------------------------------- binning (Sec. 3.1 pre-sort)
def test_oracle_tile_binning_counts_and_order():
    """P7 (oracle side): every record is listed in exactly the tiles of its tile
    rectangle (count = closed form (x1//t - x0//t + 1)(y1//t - y0//t + 1)), each
    tile's list is sorted by (depth bits, record index), and the ranges cover it."""
    rng = np.random.default_rng(5)
    n, t = 500, 16
    cam = synth.Camera(200, 120, 1, 1, 0, 0)
    x0 = rng.integers(0, 200, n)
    y0 = rng.integers(0, 120, n)
    rect = np.c_[x0, y0, np.minimum(199, x0 + rng.integers(0, 40, n)), np.minimum(119, y0 + rng.integers(0, 40, n))]
    rect[::17] = [1, 1, 0, 0]  # culled
    depth = rng.choice(np.float32([0.5, 1.0, 2.0, 3.0]), n)  # many exact ties
    keys, vals, ranges = oracle.bin_tiles(rect, depth, n, t, [cam])
    cnt = np.bincount(vals, minlength=n)
    want = np.where(rect[:, 0] > rect[:, 2], 0,
                    (rect[:, 2] // t - rect[:, 0] // t + 1) * (rect[:, 3] // t - rect[:, 1] // t + 1))
    assert np.array_equal(cnt, want)
    tiles = (keys >> np.uint64(32)).astype(np.int64)
    for tid in range(ranges.shape[0]):
        a, b = ranges[tid]
        assert np.all(tiles[a:b] == tid)
        zb = (keys[a:b] & np.uint64(0xFFFFFFFF)).astype(np.int64)
        order = np.lexsort((vals[a:b], zb))
        assert np.array_equal(order, np.arange(b - a))
    assert ranges[:, 1].max() == len(keys)


# ----------------------------------------------------------- pose update
def test_adam_first_step_is_signed_learning_rate():
    """Adam's first step has mhat = g, vhat = g^2, so each coordinate moves by
    -lr * sign(g) (Sec. 4 learning rates {0.0015 rot, 0.00215 trans}); the rotation
    part stays orthonormal."""
    st = np.zeros(25)
    st[:9] = np.eye(3).reshape(-1)
    st[9:12] = [0.3, -0.2, 1.0]
    g = np.array([2.0, -3.0, 0.5, 0.0, 0.0, 0.0])
    oracle.adam_step(st, g, lr_rot=0.0015, lr_trans=0.00215, eps=1e-12)
    np.testing.assert_allclose(st[9:12], [0.3 - 0.00215, -0.2 + 0.00215, 1.0 - 0.00215], rtol=0, atol=1e-12)
    # rotation-only gradient about z (t = 0 so the {so(3)|T} conversion is the identity)
    st = np.zeros(25)
    st[:9] = np.eye(3).reshape(-1)
    oracle.adam_step(st, np.array([0, 0, 0, 0, 0, -1.0]), eps=1e-12)
    th = 0.0015
    want = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    np.testing.assert_allclose(st[:9].reshape(3, 3), want, atol=1e-15)


def _exp_so3(w):
    """Rotation matrix of the rotation vector w (scipy's Rodrigues, a library
    routine independent of the oracle's own exponential)."""
    from scipy.spatial.transform import Rotation
    return Rotation.from_rotvec(np.asarray(w, float)).as_matrix()


def _log_so3(R):
    from scipy.spatial.transform import Rotation
    return Rotation.from_matrix(R).as_rotvec()


def test_pose_update_gradient_conversion_by_finite_differences():
    """Sec. 3.4 (pose as {so(3) | T}, R <- Exp(dR) R, t <- t + dt): the Adam step
    turns the left-perturbation gradient (g_rho, g_phi) of T(xi) = Exp(xi) T_cw
    into the gradient of the paper's parameters (dR, dt). Both gradients are
    taken here by central differences of one toy loss L(R, t) of a rigid point
    set, each in its own parametrisation; with a large Adam epsilon the first
    step is d = -lr g / (|g| + eps), which is inverted exactly to read back the
    converted gradient the oracle used. t is far from 0, so the conversion is
    not the identity (it differs from g_phi by several times the tolerance)."""
    rng = np.random.default_rng(11)
    pts = rng.normal(size=(7, 3))
    c = rng.normal(size=3)
    Aq = rng.normal(size=(3, 3))
    Aq = Aq @ Aq.T

    def loss(R, t):
        x = pts @ R.T + t
        return float(np.sum(x @ c) + 0.5 * np.einsum("ni,ij,nj->", x, Aq, x) + np.sum(np.sin(x[:, 0] * x[:, 1])))

    R0 = _exp_so3([0.4, -0.9, 0.3])
    t0 = np.array([0.7, -0.4, 1.3])
    h = 1e-6
    E = np.eye(3)
    g_rho = np.array([(loss(R0, t0 + h * E[k]) - loss(R0, t0 - h * E[k])) / (2 * h) for k in range(3)])
    g_phi = np.array([(loss(_exp_so3(h * E[k]) @ R0, _exp_so3(h * E[k]) @ t0)
                       - loss(_exp_so3(-h * E[k]) @ R0, _exp_so3(-h * E[k]) @ t0)) / (2 * h) for k in range(3)])
    G_t = np.array([(loss(R0, t0 + h * E[k]) - loss(R0, t0 - h * E[k])) / (2 * h) for k in range(3)])
    G_R = np.array([(loss(_exp_so3(h * E[k]) @ R0, t0) - loss(_exp_so3(-h * E[k]) @ R0, t0)) / (2 * h)
                    for k in range(3)])
    assert np.abs(G_R - g_phi).max() > 1e3 * 1e-7 * np.abs(G_R).max()  # t really matters

    st = np.zeros(25)
    st[:9] = R0.reshape(-1)
    st[9:12] = t0
    lr, eps = 1.0, 1e3
    oracle.adam_step(st, np.r_[g_rho, g_phi], lr_rot=lr, lr_trans=lr, eps=eps)
    d_t = st[9:12] - t0
    d_R = _log_so3(st[:9].reshape(3, 3) @ R0.T)

    def used(d):  # invert d = -lr g / (|g| + eps)
        r = -np.asarray(d) / lr
        return eps * r / (1 - np.abs(r))

    scale = max(np.abs(G_t).max(), np.abs(G_R).max())
    np.testing.assert_allclose(used(d_t), G_t, rtol=0, atol=1e-7 * scale)
    np.testing.assert_allclose(used(d_R), G_R, rtol=0, atol=1e-7 * scale)


def test_pose_update_rotation_step_from_translation_gradient():
    """Sec. 3.4: with t = (1, 0, 0), g_phi = 0 and g_rho = (0, 1, 0) (the loss
    grows as the left perturbation moves points along +y), rotate the pose by a
    small angle d about z in the paper's parameters, R <- Exp(d e_z) R with t
    held. In the left perturbation Exp(xi) T that is phi = d e_z together with
    rho = -phi x t = (0, -d, 0), since Exp(phi) would otherwise also turn t to
    (1, d, 0). The loss therefore changes by g_rho . rho = -d: the rotation
    gradient about z is -1 (hand-derived), and x and y are 0. Adam's first step
    is -lr sign(g): t_y decreases by lr_trans and the pose rotates by +lr_rot
    about z."""
    st = np.zeros(25)
    st[:9] = np.eye(3).reshape(-1)
    st[9:12] = [1.0, 0.0, 0.0]
    oracle.adam_step(st, np.array([0, 1.0, 0, 0, 0, 0]), lr_rot=0.0015, lr_trans=0.00215, eps=1e-12)
    th = 0.0015
    want = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    np.testing.assert_allclose(st[:9].reshape(3, 3), want, rtol=0, atol=1e-14)
    np.testing.assert_allclose(st[9:12], [1.0, -0.00215, 0.0], rtol=0, atol=1e-14)


def test_adam_moments_over_three_steps_closed_form():
    """Adam (Sec. 4 learning rates, beta = (0.9, 0.999)) over gradients g, -g, g:
    m_1 = (1-b1) g, m_2 = -(1-b1)^2 g, m_3 = (1-b1)(1-b1+b1^2) g and
    v_k = (1-b2^k) g^2, so the bias-corrected steps are -lr g/(|g|+eps) times 1,
    -(1-b1)/(1+b1) and (1-b1+b1^2)/(1+b1+b1^2) (hand-derived sums of the
    geometric recursions). t stays parallel to g_rho = (s, s, s), so the
    rotation gradient is g_phi at every step; the pose after three steps is the
    product of the three rotation steps (scipy's exponential) and the sum of the
    translation steps."""
    b1, b2, eps, lr_r, lr_t = 0.9, 0.999, 1e-8, 0.0015, 0.00215
    g = np.array([0.02, 0.02, 0.02, 0.3, -1.7, 0.05])
    st = np.zeros(25)
    R0 = _exp_so3([0.1, 0.2, -0.3])
    st[:9] = R0.reshape(-1)
    t0 = np.array([0.5, 0.5, 0.5])
    st[9:12] = t0
    for k, s in enumerate((1, -1, 1)):
        oracle.adam_step(st, s * g, lr_rot=lr_r, lr_trans=lr_t, beta1=b1, beta2=b2, eps=eps)
    assert st[24] == 3
    np.testing.assert_allclose(st[12:18], (1 - b1) * (1 - b1 + b1 * b1) * g, rtol=1e-13, atol=0)
    np.testing.assert_allclose(st[18:24], (1 - b2 ** 3) * g * g, rtol=1e-13, atol=0)
    unit = g / (np.abs(g) + eps)
    f = [1.0, -(1 - b1) / (1 + b1), (1 - b1 + b1 * b1) / (1 + b1 + b1 * b1)]
    lr = np.r_[[lr_t] * 3, [lr_r] * 3]
    d = [-lr * fk * unit for fk in f]
    np.testing.assert_allclose(st[9:12], t0 + d[0][:3] + d[1][:3] + d[2][:3], rtol=0, atol=1e-15)
    R = _exp_so3(d[2][3:]) @ _exp_so3(d[1][3:]) @ _exp_so3(d[0][3:]) @ R0
    np.testing.assert_allclose(st[:9].reshape(3, 3), R, rtol=0, atol=1e-14)
