"""Pins of the oracle's pseudo-normal, normal loss (Sec. 4.3, Eq. 23-25) and training-stage
transfer (Sec. 4.5, Eq. 28) against closed forms, independent quadrature and limits (CPU)."""
import math

import numpy as np
import pytest
import torch

from oracle import render as R
from paper_2408_03538_gb300 import scenes as S


def _cam64(eye, target, fov, w, h):
    """look_at_camera with its rotation and translation kept in FP64."""
    c = S.look_at_camera(eye, target, fov, w, h)
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, [0.0, 0.0, 1.0])
    r /= np.linalg.norm(r)
    rot = np.stack([r, np.cross(f, r), f])
    fy = 0.5 * h / math.tan(math.radians(fov) / 2)
    return S.Camera(rot=rot, trans=-rot @ eye, fx=fy, fy=fy, cx=c.cx, cy=c.cy, width=w, height=h, near=c.near,
                    position=eye)


def _rays(cam):
    """World-space origin and per-pixel ray directions (camera z = 1) of a pinhole camera."""
    W, H = cam.width, cam.height
    R_ = np.asarray(cam.rot, np.float64)
    eye = -R_.T @ np.asarray(cam.trans, np.float64)
    u = (np.arange(W) - cam.cx) / cam.fx
    v = (np.arange(H) - cam.cy) / cam.fy
    rc = np.stack([np.broadcast_to(u[None, :], (H, W)), np.broadcast_to(v[:, None], (H, W)), np.ones((H, W))], -1)
    return eye, rc @ R_  # rows: R^T rc


def _plane_depth(cam, p0, nrm):
    eye, d = _rays(cam)
    s = (nrm @ (p0 - eye)) / (d @ nrm)
    return np.where(s > 0, s, 0.0)


def _sphere_depth(cam, c, rho):
    eye, d = _rays(cam)
    oc = eye - c
    a = np.einsum("hwk,hwk->hw", d, d)
    b = 2 * d @ oc
    cc = oc @ oc - rho * rho
    disc = b * b - 4 * a * cc
    s = (-b - np.sqrt(np.maximum(disc, 0))) / (2 * a)
    return np.where(disc > 0, s, 0.0)


# ------------------------------------------------------------------------------------------
# Pseudo-normal (Eq. 24)
# ------------------------------------------------------------------------------------------
def test_backproject_inverts_the_projection():
    """backproject(depth) lands on points whose projection (u = fx x/z + cx, as in
    preprocess) is the pixel and whose camera-space z is the depth."""
    cam = _cam64((1.0, -5.0, 2.0), (0.2, 0.1, 0.3), 50, 40, 30)
    D = np.random.default_rng(1).uniform(1, 3, (30, 40))
    X = R.backproject(D, cam)
    Xc = X @ np.asarray(cam.rot).T + np.asarray(cam.trans)
    np.testing.assert_allclose(Xc[..., 2], D, rtol=1e-13)
    np.testing.assert_allclose(cam.fx * Xc[..., 0] / Xc[..., 2] + cam.cx, np.arange(40)[None, :] + 0 * D,
                               atol=1e-10)
    np.testing.assert_allclose(cam.fy * Xc[..., 1] / Xc[..., 2] + cam.cy, np.arange(30)[:, None] + 0 * D,
                               atol=1e-10)


@pytest.mark.parametrize("nrm", [(0.0, 0.0, 1.0), (-0.3, 0.2, 1.0), (0.5, -1.0, 0.4)])
def test_pseudo_normal_of_a_plane_is_its_normal(nrm):
    """Central differences of back-projected points of a plane lie in the plane, so N' is the
    plane's normal exactly (to rounding), oriented toward the camera, at every pixel."""
    cam = _cam64((0.5, -6.0, 3.0), (0.0, 0.0, 0.0), 20, 48, 36)
    nrm = np.asarray(nrm, np.float64)
    nrm /= np.linalg.norm(nrm)
    D = _plane_depth(cam, np.zeros(3), nrm)
    assert np.all(D > 0)
    N = R.pseudo_normal(D, cam)
    eye = np.asarray(cam.position, np.float64)
    facing = nrm if nrm @ eye > 0 else -nrm
    inner = N[:, 1:-1, 1:-1].reshape(3, -1)
    np.testing.assert_allclose(inner, np.repeat(facing[:, None], inner.shape[1], 1), atol=1e-10)
    assert np.all(N[:, 0] == 0) and np.all(N[:, -1] == 0) and np.all(N[:, :, 0] == 0) and np.all(N[:, :, -1] == 0)


def _sphere_err(w):
    cam = _cam64((0.0, -4.0, 1.0), (0.0, 0.0, 0.0), 30, w, w)
    c, rho = np.array([0.1, 0.0, -0.05]), 0.8
    D = _sphere_depth(cam, c, rho)
    N = R.pseudo_normal(D, cam)
    X = R.backproject(D, cam)
    ref = (X - c) / rho
    eye = np.asarray(cam.position, np.float64)
    view = eye - X
    view /= np.maximum(np.linalg.norm(view, axis=-1, keepdims=True), 1e-300)
    sel = (np.einsum("hwk,hwk->hw", ref, view) > 0.5) & np.any(N != 0, axis=0)
    assert sel.sum() > 100
    err = np.linalg.norm(np.moveaxis(N, 0, -1)[sel] - ref[sel], axis=-1)
    return float(err.max())


def test_pseudo_normal_of_a_sphere_is_second_order():
    """On a sphere N' tends to the analytic normal (X - c)/rho; central differences make the
    error fall ~4x when the pixel pitch halves (a one-sided difference would give 2x)."""
    e1, e2, e3 = _sphere_err(64), _sphere_err(128), _sphere_err(256)
    assert e1 < 2e-2
    assert e2 / e1 < 0.3 and e3 / e2 < 0.3


def test_pseudo_normal_rotates_with_the_world():
    """Rotating the scene and the camera together leaves the depth map unchanged and rotates
    N' by the same rotation (world-space output)."""
    cam = _cam64((0.0, -4.0, 1.0), (0.0, 0.0, 0.0), 35, 40, 32)
    D = _sphere_depth(cam, np.array([0.0, 0.1, 0.0]), 0.9)
    N = R.pseudo_normal(D, cam)
    th = 0.7
    ax = np.array([1.0, 2.0, -0.5])
    ax /= np.linalg.norm(ax)
    K = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
    Q = np.eye(3) + math.sin(th) * K + (1 - math.cos(th)) * K @ K
    rot2 = np.asarray(cam.rot) @ Q.T
    eye2 = Q @ np.asarray(cam.position)
    cam2 = S.Camera(rot=rot2, trans=-rot2 @ eye2, fx=cam.fx, fy=cam.fy, cx=cam.cx, cy=cam.cy, width=cam.width,
                    height=cam.height, near=cam.near, position=eye2)
    N2 = R.pseudo_normal(D, cam2)
    np.testing.assert_allclose(N2, np.einsum("ab,bhw->ahw", Q, N), atol=1e-12)
    assert np.abs(N).max() > 0.5


def test_pseudo_normal_undefined_where_a_neighbour_has_no_depth():
    cam = _cam64((0.0, -4.0, 1.0), (0.0, 0.0, 0.0), 35, 12, 10)
    D = _plane_depth(cam, np.zeros(3), np.array([0.0, 0.0, 1.0]))
    D[4, 6] = 0.0
    N = R.pseudo_normal(D, cam)
    zero = np.all(N == 0, axis=0)
    for (y, x) in [(4, 6), (3, 6), (5, 6), (4, 5), (4, 7)]:
        assert zero[y, x]
    assert not zero[3, 5] and not zero[2, 6]
    np.testing.assert_allclose(np.linalg.norm(N[:, ~zero], axis=0), 1.0, rtol=1e-12)
    assert R.pseudo_normal(np.ones((2, 5)), cam).shape == (3, 2, 5)
    assert np.all(R.pseudo_normal(np.ones((2, 5)), cam) == 0)


def test_pseudo_normal_of_a_splat_plane_follows_the_plane():
    """Eq. 23 then Eq. 24: the depth composite of a dense tilted plane of flat splats gives a
    pseudo-normal close to the plane's normal. D blends the depths of the splat centres in
    front-to-back order, so it is the plane only up to a small staircase; the median angle
    and the 90th percentile are what is held."""
    rng = np.random.default_rng(3)
    th = -math.atan(0.3)  # plane z = 0.3 x: normal (-0.3, 0, 1)/|.|, e_z turned about y by th
    nrm = np.array([math.sin(th), 0.0, math.cos(th)])
    u = rng.uniform(-1.2, 1.2, (10000, 2))
    e1 = np.array([math.cos(th), 0.0, -math.sin(th)])
    e2 = np.array([0.0, 1.0, 0.0])
    means = u[:, :1] * e1 + u[:, 1:] * e2
    n = means.shape[0]
    scales = np.tile([0.03, 0.03, 0.0006], (n, 1))
    quats = np.tile([math.cos(th / 2), 0.0, math.sin(th / 2), 0.0], (n, 1))
    cam = _cam64((-0.6, -1.2, 2.9), (0.0, 0.0, 0.0), 25, 32, 24)
    Rw = np.asarray(cam.rot)
    d = means @ Rw[2] + cam.trans[2]
    feats = np.zeros((1, n, 3))
    feats[0, :, 0] = d
    t = lambda a: torch.as_tensor(np.asarray(a, np.float64))
    D = R.render(t(means), t(scales), t(quats), t(np.full(n, 0.9)), t(feats), cam).numpy()[0, 0]
    N = R.pseudo_normal(D, cam)
    facing = nrm if nrm @ np.asarray(cam.position) > 0 else -nrm
    c = N[:, 1:-1, 1:-1].reshape(3, -1)
    assert np.all(np.abs(np.linalg.norm(c, axis=0) - 1) < 1e-12)  # defined everywhere inside
    ang = np.degrees(np.arccos(np.clip(facing @ c, -1, 1)))
    assert float(np.median(ang)) < 2.0 and float(np.percentile(ang, 90)) < 4.0
    # the transposed rotation would put the normal elsewhere
    wrong = np.asarray(cam.rot) @ facing
    assert float(np.median(np.degrees(np.arccos(np.clip(wrong @ c, -1, 1))))) > 20.0


# ------------------------------------------------------------------------------------------
# Normal loss (Eq. 25)
# ------------------------------------------------------------------------------------------
def _unit_map(rng, h, w):
    m = rng.normal(size=(3, h, w))
    return m / np.linalg.norm(m, axis=0, keepdims=True)


def test_normal_loss_definition():
    rng = np.random.default_rng(4)
    Np = _unit_map(rng, 6, 7)
    Np[:, 0, :] = 0.0  # undefined pixels
    L, g = R.normal_loss(Np, Np)
    assert L == 0.0 and np.all(g == 0)
    N = Np.copy()
    N[:, 3, 2] += np.array([0.0, 0.6, -0.8])  # one pixel off by a unit vector x 1
    L, g = R.normal_loss(N, Np)
    assert L == pytest.approx(1.0, rel=1e-14)
    np.testing.assert_allclose(g[:, 3, 2], [0.0, 0.6, -0.8], rtol=1e-14)
    N[:, 0, :] = 5.0  # a difference where N' is undefined does not count
    assert R.normal_loss(N, Np)[0] == pytest.approx(1.0, rel=1e-14)
    D = rng.normal(size=Np.shape)
    D[:, 0, :] = 0
    assert R.normal_loss(Np + 3 * D, Np)[0] == pytest.approx(3 * R.normal_loss(Np + D, Np)[0], rel=1e-13)


def test_normal_loss_gradient_central_differences():
    rng = np.random.default_rng(5)
    Np = _unit_map(rng, 5, 4)
    Np[:, 2, 1] = 0.0
    N = _unit_map(rng, 5, 4)
    L, g = R.normal_loss(N, Np)
    h = 1e-6
    num = np.zeros_like(N)
    for idx in np.ndindex(N.shape):
        Nh = N.copy()
        Nh[idx] += h
        Nl = N.copy()
        Nl[idx] -= h
        num[idx] = (R.normal_loss(Nh, Np)[0] - R.normal_loss(Nl, Np)[0]) / (2 * h)
    np.testing.assert_allclose(g, num, atol=1e-8)
    assert np.all(g[:, 2, 1] == 0)


# ------------------------------------------------------------------------------------------
# Training-stage transfer (Eq. 28)
# ------------------------------------------------------------------------------------------
def _occluded_scene(n=60, seed=7):
    sc = S.isotropic_scene(n, seed)
    rng = np.random.default_rng(seed)
    sc.roughness = rng.uniform(0.2, 0.9, n)
    sc.metallic = rng.uniform(0.0, 0.8, n)
    return sc


def test_training_transfer_without_specular_is_the_diffuse_transfer(oracle_mod):
    """Eq. 28 with f_s = 0 is f_d (w.n) V (Eq. 29): with k = 1 - m the training transfer is
    (1 - m) P, P from the C oracle's shadowed transfer of the same receivers."""
    sc = _occluded_scene()
    dirs = S.direction_set(96, 2)
    recv = np.arange(0, 60, 3)
    tr = oracle_mod.transfer(sc, dirs, 3, recv)
    cam_pos = np.array([0.3, -4.0, 1.5])
    t = oracle_mod.training_transfer(sc, dirs, 3, recv, tr["V"], cam_pos, specular=False)
    v = oracle_mod.view_dirs(sc.means[recv], cam_pos)
    front = np.einsum("rk,rk->r", v, sc.normals[recv] / np.linalg.norm(sc.normals[recv], axis=1, keepdims=True)) > 0
    ref = (1.0 - sc.metallic[recv])[:, None] * tr["P"] * front[:, None]
    np.testing.assert_allclose(t, ref, atol=1e-12)
    assert front.sum() >= 5 and (~front).sum() >= 3
    assert np.any(tr["V"][front] < 0.999)  # the receivers are occluded


def _hemisphere_gl(nth, nph):
    x, w = np.polynomial.legendre.leggauss(nth)
    th = (x + 1) * math.pi / 4  # [0, pi/2]
    wth = w * math.pi / 4
    xp, wp = np.polynomial.legendre.leggauss(nph)
    ph = (xp + 1) * math.pi
    wph = wp * math.pi
    T, P = np.meshgrid(th, ph, indexing="ij")
    d = np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], -1).reshape(-1, 3)
    wt = (wth[:, None] * wph[None, :] * np.sin(T)).reshape(-1)
    return d, wt


@pytest.mark.parametrize("r,m,vth", [(0.6, 0.2, 0.7), (0.9, 0.0, 1.2), (0.45, 0.5, 0.3)])
def test_training_transfer_unoccluded_is_the_brdf_cosine_integral(oracle_mod, r, m, vth):
    """V = 1: t[c] tends to int k(w, v) (n.w)^+ Y_c(w) dw over the sphere of incident
    directions. The reference integral is a Gauss-Legendre product rule over the upper
    hemisphere, independent of the direction set; reading the cosine as (v.n) (the printed
    form) or taking Y at v would change the result by far more than the tolerance."""
    n = np.array([0.0, 0.0, 1.0])
    sc = S._finish(np.zeros((1, 3)), np.full((1, 3), 0.05), np.array([[1.0, 0, 0, 0]]), np.array([0.5]), n[None],
                   np.full((1, 3), 0.5), roughness=np.array([r]), metallic=np.array([m]))
    cam_pos = 10.0 * np.array([math.sin(vth), 0.3 * math.sin(vth), math.cos(vth)])
    v = cam_pos / np.linalg.norm(cam_pos)
    dirs = S.direction_set(1 << 17, 9).astype(np.float64)
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    t = oracle_mod.training_transfer(sc, dirs, 2, [0], np.ones((1, dirs.shape[0])), cam_pos)[0]
    gd, gw = _hemisphere_gl(160, 320)
    k = oracle_mod.brdf_kernel(n[None], gd, v[None], r, m)
    ref = (gw * k * gd[:, 2]) @ oracle_mod.sh(2, gd)
    np.testing.assert_allclose(t, ref, atol=3e-3 * abs(ref[0]))
    wrong_cos = (gw * k * (v @ n)) @ oracle_mod.sh(2, gd)
    assert np.abs(wrong_cos - ref).max() > 0.05 * abs(ref[0])


def test_training_transfer_zero_behind_the_view_and_linear_in_V(oracle_mod):
    sc = _occluded_scene(20, 11)
    dirs = S.direction_set(64, 3)
    rng = np.random.default_rng(0)
    V1 = rng.uniform(0, 1, (20, 64))
    V2 = rng.uniform(0, 1, (20, 64))
    cam = np.array([1.0, -3.0, 2.0])
    t1 = oracle_mod.training_transfer(sc, dirs, 3, np.arange(20), V1, cam)
    t2 = oracle_mod.training_transfer(sc, dirs, 3, np.arange(20), V2, cam)
    t12 = oracle_mod.training_transfer(sc, dirs, 3, np.arange(20), V1 + 2 * V2, cam)
    np.testing.assert_allclose(t12, t1 + 2 * t2, atol=1e-12)
    v = oracle_mod.view_dirs(sc.means, cam)
    back = np.einsum("rk,rk->r", v, sc.normals) <= 0
    assert back.any() and (~back).any()
    assert np.all(t1[back] == 0) and np.all(np.abs(t1[~back]).sum(1) > 0)


def test_training_transfer_gradient_complex_step_matches_central_differences(oracle_mod):
    sc = _occluded_scene(12, 13)
    dirs = S.direction_set(64, 4)
    recv = np.arange(12)
    rng = np.random.default_rng(2)
    V = rng.uniform(0.2, 1, (12, 64))
    cam = np.array([0.5, -3.0, 1.0])
    dT = rng.normal(size=(12, 16))
    gr, gm = oracle_mod.training_transfer_grad(sc, dirs, 3, recv, V, cam, dT)
    h = 1e-6
    r0, m0 = sc.roughness.copy(), sc.metallic.copy()
    f = lambda rr, mm: (dT * oracle_mod.training_transfer(sc, dirs, 3, recv, V, cam, roughness=rr,
                                                          metallic=mm)).sum(1)
    num_r = (f(r0 + h, m0) - f(r0 - h, m0)) / (2 * h)
    num_m = (f(r0, m0 + h) - f(r0, m0 - h)) / (2 * h)
    np.testing.assert_allclose(gr, num_r, rtol=1e-6, atol=1e-8)
    np.testing.assert_allclose(gm, num_m, rtol=1e-6, atol=1e-8)
    assert np.abs(gr).max() > 1e-3 and np.abs(gm).max() > 1e-3
