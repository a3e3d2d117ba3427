"""Pins of the oracle's analytic FP64 adjoint (the backward of Eq. 1-10 and the
se(3) pose gradient of Sec. 3.4) against central finite differences and against
rigid-motion invariants that tie the pose gradient to the parameter gradients.

Finite differences skip any element whose perturbation changes a discrete
decision of the blend (membership q <= 9, alpha >= 1/255, the 0.99 clamp, the
T >= 1e-4 stop): the oracle returns a hash of every decision, and only
elements with identical hashes at all stencil points are compared.
"""

import math

import numpy as np
import pytest

import oracle
import synth


def _exp_se3(xi):
    """Rotation/translation of the left increment Exp(xi) for xi = (rho, phi):
    Rodrigues for the rotation; the translation part is rho itself because the
    increment is applied as p -> R_inc p + rho (first order identical to the
    SE(3) exponential, exact derivative at xi = 0)."""
    rho, phi = np.asarray(xi[:3], float), np.asarray(xi[3:], float)
    th = np.linalg.norm(phi)
    K = np.array([[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]])
    if th == 0:
        return np.eye(3), rho
    return np.eye(3) + math.sin(th) / th * K + (1 - math.cos(th)) / th ** 2 * K @ K, rho


def _perturb_pose(T, xi):
    R, rho = _exp_se3(xi)
    out = np.zeros((3, 4))
    out[:, :3] = R @ T[:, :3]
    out[:, 3] = R @ T[:, 3] + rho
    return out


@pytest.fixture(scope="module")
def fd_case():
    sc, cam, T = synth.fd_scene()
    tc, td = synth.random_targets(cam, 1100 + 3, depth_range=(2, 4))
    L = oracle.LossSpec(1.0, 1.0, 1.0, 1.0, 0.0, tc[0], td[0])
    g = oracle.grad(sc, cam, T, L)
    base, h0 = oracle.loss_value(sc, cam, T, L)
    return sc, cam, T, L, g, base, h0


def test_loss_value_matches_between_entry_points(fd_case):
    sc, cam, T, L, g, base, _ = fd_case
    assert abs(g["loss"] - base) <= 1e-14 * abs(base)


def test_jacobian_clamp_is_exercised(fd_case):
    """The edge Gaussians sit beyond 1.3x the half field of view in x/z yet still
    reach the image, so the clamped branch of the Jacobian is covered."""
    sc, cam, T, *_ = fd_case
    pr = oracle.project(sc, cam, T)
    xz = np.abs(sc.means[:, 0] / sc.means[:, 2])
    lim = 1.3 * 0.5 * cam.width / cam.fx
    assert np.any(pr["valid"] & (xz > lim))


@pytest.mark.parametrize("field,dim", [("means", 3), ("log_scales", 3), ("quats", 4),
                                       ("opacity_logit", 1), ("colors", 3), ("nu", 1)])
def test_parameter_gradients_match_central_differences(fd_case, field, dim):
    """P8: 4-point central differences (h = 1e-5) of the FP64 loss agree with the
    analytic gradient to 1e-6 relative on every element whose decisions are
    stable, above an absolute floor set by FP64 rounding of the loss."""
    sc, cam, T, L, g, base, h0 = fd_case
    h = 1e-5
    floor = 1e3 * np.finfo(float).eps * abs(base) / h
    arr = getattr(sc, field)
    n_checked = 0
    for i in range(sc.n):
        for c in range(dim):
            idx = (i, c) if arr.ndim == 2 else (i,)
            old = arr[idx]
            vals = []
            ok = True
            for s in (-2, -1, 1, 2):
                arr[idx] = old + s * h
                v, hh = oracle.loss_value(sc, cam, T, L)
                ok &= hh == h0
                vals.append(v)
            arr[idx] = old
            if not ok:
                continue
            fd = (vals[0] - 8 * vals[1] + 8 * vals[2] - vals[3]) / (12 * h)
            an = g[field][idx]
            assert abs(fd - an) <= 1e-6 * abs(an) + floor, (field, i, c, fd, an)
            n_checked += 1
    assert n_checked >= 0.9 * sc.n * dim


def test_pose_gradient_matches_central_differences(fd_case):
    """P8 for the pose (O13): central differences of L(Exp(xi) T) at xi = 0 agree
    with the analytic left se(3) gradient (rho, phi) to 1e-6 relative. The step
    shrinks until no pixel decision changes."""
    sc, cam, T, L, g, base, h0 = fd_case
    for k in range(6):
        for h in (1e-6, 3e-7, 1e-7, 3e-8):
            xi = np.zeros(6)
            xi[k] = h
            vp, hp = oracle.loss_value(sc, cam, _perturb_pose(T, xi), L)
            vm, hm = oracle.loss_value(sc, cam, _perturb_pose(T, -xi), L)
            if hp == h0 and hm == h0:
                fd = (vp - vm) / (2 * h)
                assert abs(fd - g["pose"][k]) <= 1e-6 * abs(g["pose"][k]) + 1e2 * np.finfo(float).eps * base / h, (k, fd, g["pose"][k])
                break
        else:
            pytest.fail(f"pose component {k}: no decision-stable step found")


def _quat_mul(a, b):
    w1, v1 = a[0], np.asarray(a[1:])
    w2, v2 = b[..., 0], b[..., 1:]
    w = w1 * w2 - v2 @ v1
    v = w1 * v2 + w2[:, None] * v1[None, :] + np.cross(v1[None, :], v2)
    return np.c_[w, v]


@pytest.fixture(scope="module")
def posed_tiny():
    """Tiny scene seen from a non-identity pose so R and t both matter."""
    sc, cam, T0 = synth.tiny_scene()
    sc = synth.Scene(*(np.asarray(getattr(sc, f), np.float64) for f in
                       ("means", "log_scales", "quats", "opacity_logit", "colors", "nu")))
    T = _perturb_pose(np.asarray(T0, float), np.array([0.05, -0.03, 0.2, 0.02, -0.04, 0.03]))
    tc, td = synth.random_targets(cam, 1001 + 60)
    L = oracle.LossSpec(0.2, 1.0, 0.5, 0.5, 0.025, tc[0], td[0])
    return sc, cam, T, L, oracle.grad(sc, cam, T, L)


def test_pose_translation_equals_rotated_sum_of_mean_gradients(posed_tiny):
    """P10a: translating the camera by rho is translating every mean by -R^T rho,
    hence g_rho = R sum_i dL/dmu_i."""
    sc, cam, T, L, g = posed_tiny
    want = T[:, :3] @ g["means"].sum(0)
    np.testing.assert_allclose(g["pose"][:3], want, rtol=1e-9, atol=1e-12 * np.abs(want).max())


def test_pose_rotation_equals_scene_rotation_derivative(posed_tiny):
    """P10b: rotating the camera by Exp(phi) about its centre equals rotating every
    Gaussian (mean about the camera centre, orientation by R^T Exp(phi) R); the
    directional derivative computed from the mean and quaternion gradients must
    equal g_phi."""
    sc, cam, T, L, g = posed_tiny
    R, t = T[:, :3], T[:, 3]
    p = sc.means @ R.T + t
    got = []
    for k in range(3):
        e = np.zeros(3)
        e[k] = 1.0
        dmu = np.cross(e[None, :], p) @ R            # R^T (e x p_i), row form
        w = R.T @ e
        dq = 0.5 * _quat_mul(np.r_[0.0, w], sc.quats)
        got.append((g["means"] * dmu).sum() + (g["quats"] * dq).sum())
    np.testing.assert_allclose(g["pose"][3:], got, rtol=1e-9, atol=1e-12 * np.abs(got).max())


def test_alignment_loss_gradient_matches_central_differences():
    """f1 (Eq. 7-8, 12): L_align = mean |D_alpha - D_median| alone. D_median is
    the depth of the Gaussian at which T first drops below 0.5, so its gradient
    reaches that Gaussian's depth only; central differences of the FP64 loss
    agree with the analytic gradient (means, which move z, and the pose)."""
    sc, cam, T = synth.fd_scene()
    _, td = synth.random_targets(cam, 1100 + 4, depth_range=(2, 4))
    L = oracle.LossSpec(0.0, 0.0, 0.0, 0.0, 0.0, None, td[0], w_align=1.0)
    g = oracle.grad(sc, cam, T, L)
    base, h0 = oracle.loss_value(sc, cam, T, L)
    assert base > 0
    h = 1e-5
    floor = 1e3 * np.finfo(float).eps * abs(base) / h
    checked = 0
    for i in range(sc.n):
        for c in range(3):
            old = sc.means[i, c]
            vals, ok = [], True
            for s in (-2, -1, 1, 2):
                sc.means[i, c] = old + s * h
                v, hh = oracle.loss_value(sc, cam, T, L)
                ok &= hh == h0
                vals.append(v)
            sc.means[i, c] = old
            if not ok:
                continue
            fd = (vals[0] - 8 * vals[1] + 8 * vals[2] - vals[3]) / (12 * h)
            assert abs(fd - g["means"][i, c]) <= 1e-6 * abs(g["means"][i, c]) + floor, (i, c, fd, g["means"][i, c])
            checked += 1
    assert checked >= 0.9 * sc.n * 3
    # z of a median Gaussian moves D_median one for one: the depth row must carry it
    assert np.abs(g["g_depth"]).max() > 0
