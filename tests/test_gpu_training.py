"""GPU parity of the training-stage calls against the FP64 oracle: the visibility cache, the
training-stage view transfer and its roughness / metallic gradients (Sec. 4.5, Eq. 28), the
pseudo-normal of the depth map (Eq. 24) and the normal loss with its gradient (Eq. 25).

Tolerances. The visibility follows the transfer's allowance (|V_gpu - V_ref| <= dV + t_min +
2e-6, dV the oracle's flagged-decision bound). The view transfer is compared on the GPU's own V
(the oracle consumes the same visibility rows in FP64), so only the FP32 arithmetic of the BRDF
and the sum over S directions separates the two: ||t_gpu - t_ref|| <= 2e-4 ||t_ref|| + 1e-6 per
receiver. The pseudo-normal is compared on the same depth map; its forward error bound is a few
ulp of the terms of its closed form divided by the normal's length (see the kernel), taken as
64 eps (|a p| + |b q| + 1 + |p| + |q|) / |n| per pixel.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import render as R
from paper_2408_03538_gb300 import api, scenes as S

pytestmark = pytest.mark.gpu
EPS32 = 2.0 ** -24


def _gt(scene):
    return api.GaussianTensors.from_scene(scene)


def _brdf_scene(n, seed, shrink=0.6):
    sc = S.surface_scene(n, seed)
    sc.means *= shrink
    rng = np.random.default_rng(seed + 1)
    sc.roughness = rng.uniform(0.15, 1.0, sc.n).astype(np.float32)
    sc.metallic = rng.uniform(0.0, 1.0, sc.n).astype(np.float32)
    return sc


def _visibility(sc, dirs, order, walk=0):
    g = _gt(sc)
    st = api.Status()
    bvh = api.build_bvh(g, status=st)
    d = torch.from_numpy(dirs).cuda()
    out = api.precompute_visibility(g, bvh, d, order, status=st, walk=walk)
    torch.cuda.synchronize()
    assert st.read() == 0
    return g, bvh, d, out


@pytest.mark.parametrize("walk", [0, 1])
def test_visibility_cache_matches_oracle(walk):
    sc = _brdf_scene(3000, 21)
    dirs = S.direction_set(128, 3)
    g, bvh, d, out = _visibility(sc, dirs, 3, walk)
    V = out["V"].cpu().numpy().astype(np.float64)
    recv = np.random.default_rng(0).choice(sc.n, 160, replace=False)
    ref = oracle.transfer(sc, dirs, 3, recv)
    lim = ref["dV"] + api.DEFAULT_T_MIN + 2e-6
    err = np.abs(V[recv] - ref["V"])
    assert np.all(err <= lim), float((err - lim).max())
    facing = (np.asarray(sc.normals, np.float64)[recv] @ dirs.astype(np.float64).T) > 0
    assert np.all(V[recv][~facing] == 0)
    assert np.mean(ref["V"][facing] < 0.99) > 0.05  # the scene occludes
    # the P of the same walk is the transfer call's P
    P2 = api.precompute_transfer(g, bvh, d, 3, walk=walk)["P"]
    torch.testing.assert_close(out["P"], P2, rtol=0, atol=0)


def test_visibility_walks_agree():
    """The packet walk and the per-ray walk take their hit decisions in different FP32
    arithmetic, so they agree to 2e-6 on every ray except those with a decision inside the
    oracle's rounding band (flagged): there each walk is within the oracle's allowance."""
    sc = _brdf_scene(2000, 22)
    dirs = S.direction_set(96, 4)
    V0 = _visibility(sc, dirs, 2, 0)[3]["V"].cpu().numpy().astype(np.float64)
    V1 = _visibility(sc, dirs, 2, 1)[3]["V"].cpu().numpy().astype(np.float64)
    differ = np.abs(V0 - V1) > 2e-6
    assert differ.mean() < 2e-3
    rows = np.nonzero(differ.any(axis=1))[0]
    if rows.size:
        ref = oracle.transfer(sc, dirs, 2, rows)
        flagged = (ref["flags"] & oracle.RF_AMBIG_HIT) != 0
        assert np.all(flagged[differ[rows]])
        lim = ref["dV"] + api.DEFAULT_T_MIN + 2e-6
        for V in (V0, V1):
            assert np.all(np.abs(V[rows] - ref["V"]) <= lim)


def _tt_check(sc, dirs, order, recv, cam_pos, V):
    g = _gt(sc)
    d = torch.from_numpy(dirs).cuda()
    t = api.training_transfer(g, V, d, order, cam_pos)
    torch.cuda.synchronize()
    Vh = V.cpu().numpy().astype(np.float64)
    ref = oracle.training_transfer(sc, dirs, order, recv, Vh[recv], np.asarray(cam_pos, np.float32))
    got = t.cpu().numpy().astype(np.float64)[recv]
    err = np.linalg.norm(got - ref, axis=1)
    lim = 2e-4 * np.linalg.norm(ref, axis=1) + 1e-6
    assert np.all(err <= lim), float(np.max(err / lim))
    return got, ref


@pytest.mark.parametrize("order", [1, 3, 5])
def test_training_transfer_matches_oracle(order):
    sc = _brdf_scene(2500, 23)
    dirs = S.direction_set(128, 5)
    _, _, _, out = _visibility(sc, dirs, min(order, 3))
    cam = (0.7, -4.0, 2.2)
    recv = np.random.default_rng(1).choice(sc.n, 300, replace=False)
    got, ref = _tt_check(sc, dirs, order, recv, cam, out["V"])
    v = oracle.view_dirs(sc.means[recv], np.asarray(cam, np.float32))
    front = np.einsum("rk,rk->r", v, sc.normals[recv]) > 0
    assert front.sum() > 50 and (~front).sum() > 20
    assert np.all(got[~front] == 0)
    assert np.all(np.linalg.norm(ref[front], axis=1) > 0)


def test_training_transfer_all_receivers_and_edge_cases():
    """Every receiver of a small scene; one Gaussian; a camera on a splat's tangent plane."""
    sc = _brdf_scene(700, 24)
    dirs = S.direction_set(64, 6)
    _, _, _, out = _visibility(sc, dirs, 2)
    _tt_check(sc, dirs, 2, np.arange(sc.n), (0.0, -3.0, 1.0), out["V"])
    one = S._finish(np.array([[0.2, -0.1, 0.3]]), np.full((1, 3), 0.05), np.array([[1.0, 0, 0, 0]]),
                    np.array([0.8]), np.array([[0.0, 0.0, 1.0]]), np.full((1, 3), 0.5), roughness=np.array([0.4]),
                    metallic=np.array([0.3]))
    _, _, _, o1 = _visibility(one, dirs, 2)
    assert torch.all(o1["V"][0][torch.from_numpy(dirs[:, 2] > 0).cuda()] == 1)
    _tt_check(one, dirs, 2, [0], (0.3, 0.2, 5.0), o1["V"])
    t = api.training_transfer(_gt(one), o1["V"], torch.from_numpy(dirs).cuda(), 2,
                              tuple(np.asarray(one.means[0], np.float64) + [1.0, 0.0, 0.0]))
    assert torch.all(t == 0)  # the view lies in the tangent plane: n.v = 0


def test_training_transfer_gradients_match_complex_step():
    sc = _brdf_scene(1500, 26)
    dirs = S.direction_set(128, 7)
    g, _, d, out = _visibility(sc, dirs, 3)
    cam = (-1.0, -3.5, 2.0)
    rng = np.random.default_rng(2)
    dt = rng.normal(size=(sc.n, 16)).astype(np.float32)
    dr, dm = api.training_transfer_backward(g, out["V"], d, 3, cam, torch.from_numpy(dt).cuda())
    torch.cuda.synchronize()
    recv = rng.choice(sc.n, 200, replace=False)
    Vh = out["V"].cpu().numpy().astype(np.float64)[recv]
    gr, gm = oracle.training_transfer_grad(sc, dirs, 3, recv, Vh, np.asarray(cam, np.float32), dt[recv])
    sr = np.abs(gr).max()
    sm = np.abs(gm).max()
    np.testing.assert_allclose(dr.cpu().numpy()[recv], gr, atol=2e-4 * sr, rtol=2e-4)
    np.testing.assert_allclose(dm.cpu().numpy()[recv], gm, atol=2e-5 * sm, rtol=2e-5)
    assert sr > 1e-3 and sm > 1e-3


def test_training_transfer_full_size_sampled():
    """Tiled 1M-Gaussian scene (10 copies of a 100k surface scene), order 3, S = 256: the visibility
    cache and the view transfer at full size, 256 sampled receivers against the oracle."""
    sc = S.make_scene("tiled-1m-glossy")
    dirs = S.direction_set(256, S.config_seed(2))
    g, _, d, out = _visibility(sc, dirs, 3)
    cam = S.make_camera("tiled-1m-glossy").position
    recv = np.sort(np.random.default_rng(3).choice(sc.n, 256, replace=False))
    ref = oracle.transfer(sc, dirs, 3, recv)
    V = out["V"].cpu().numpy()[recv].astype(np.float64)
    assert np.all(np.abs(V - ref["V"]) <= ref["dV"] + api.DEFAULT_T_MIN + 2e-6)
    _tt_check(sc, dirs, 3, recv, tuple(np.asarray(cam, np.float64)), out["V"])


# ---- pseudo-normal and normal loss ---------------------------------------------------------
def _pn_bound(depth, cam):
    """Per-pixel bound of the kernel's FP32 rounding (see the module docstring)."""
    D = np.asarray(depth, np.float64)
    H, W = D.shape
    out = np.zeros((H, W))
    dl, dr = D[1:-1, :-2], D[1:-1, 2:]
    du, dd = D[:-2, 1:-1], D[2:, 1:-1]
    with np.errstate(divide="ignore", invalid="ignore"):
        p = cam.fx * (dr - dl) / (dr + dl)
        q = cam.fy * (dd - du) / (dd + du)
        a = (np.arange(1, W - 1)[None, :] - cam.cx) / cam.fx
        b = (np.arange(1, H - 1)[:, None] - cam.cy) / cam.fy
        nz = -(a * p + b * q + 1)
        ln = np.sqrt(p * p + q * q + nz * nz)
        out[1:-1, 1:-1] = 64 * EPS32 * (np.abs(a * p) + np.abs(b * q) + 1 + np.abs(p) + np.abs(q)) / ln
    return np.nan_to_num(out, nan=0.0, posinf=0.0)


def _check_pn(depth_t, cam):
    got = api.pseudo_normal(depth_t, cam).cpu().numpy().astype(np.float64)
    D = depth_t.cpu().numpy().astype(np.float64)
    ref = R.pseudo_normal(D, cam)
    np.testing.assert_array_equal(np.any(got != 0, axis=0), np.any(ref != 0, axis=0))
    err = np.linalg.norm(got - ref, axis=0)
    lim = _pn_bound(D, cam) + 1e-7
    assert np.all(err <= lim), float(np.max(err / lim))
    return got, ref


def test_pseudo_normal_of_rendered_depth_matches_oracle():
    """Depth of a rendered surface scene (prtgs_render_geometry), then N' on the GPU and in FP64
    on the same depth map: the same pixels defined, values within the rounding bound."""
    sc = S.surface_scene(4000, 27)
    sc.means *= 0.5
    cam = S.look_at_camera((0.4, -4.0, 2.0), (0, 0, 0.4), 45, 200, 150)
    depth, normal, _ = api.render_geometry(_gt(sc), cam)
    got, ref = _check_pn(depth, cam)
    defined = np.any(ref != 0, axis=0)
    assert 0.2 < defined.mean() < 0.98
    # N' faces the camera wherever it is defined
    X = R.backproject(depth.cpu().numpy(), cam)
    view = np.asarray(cam.position, np.float64) - X
    assert np.all(np.einsum("khw,hwk->hw", got, view)[defined] > 0)


def test_pseudo_normal_plane_and_edges():
    """An analytic tilted-plane depth map gives the plane normal; image borders, holes, a
    one-pixel-wide image and an empty image are handled."""
    cam = S.look_at_camera((0.5, -6.0, 3.0), (0, 0, 0), 20, 67, 45)
    R64 = np.asarray(cam.rot, np.float64)
    eye = np.asarray(cam.position, np.float64)
    nrm = np.array([-0.3, 0.2, 1.0])
    nrm /= np.linalg.norm(nrm)
    u = (np.arange(67) - cam.cx) / cam.fx
    v = (np.arange(45) - cam.cy) / cam.fy
    rc = np.stack([np.broadcast_to(u[None, :], (45, 67)), np.broadcast_to(v[:, None], (45, 67)),
                   np.ones((45, 67))], -1)
    rw = rc @ R64
    s = -(eye @ nrm) / (rw @ nrm)
    D = s.astype(np.float32)
    D[10, 20] = 0.0
    D[30, 40] = -1.0
    got, _ = _check_pn(torch.from_numpy(D).cuda(), cam)
    facing = nrm if nrm @ eye > 0 else -nrm
    m = np.any(got != 0, axis=0)
    assert not m[10, 20] and not m[9, 20] and not m[30, 41] and not m[0, 5] and not m[44, 5]
    assert m.sum() == (65 * 43 - 10)
    assert np.max(np.linalg.norm(got[:, m] - facing[:, None], axis=0)) < 5e-4  # FP32 depth rounding
    thin = S.look_at_camera((0.5, -6.0, 3.0), (0, 0, 0), 20, 1, 45)
    assert torch.all(api.pseudo_normal(torch.ones((45, 1), device="cuda"), thin) == 0)


def test_pseudo_normal_full_hd():
    """1920 x 1080 depth of the tiled 1M scene from its bench camera: every pixel against the
    oracle on the same depth map."""
    sc = S.make_scene("tiled-1m-glossy")
    cam = S.make_camera("tiled-1m-glossy")
    depth, _, _ = api.render_geometry(_gt(sc), cam, max_pairs=40_000_000)
    got, ref = _check_pn(depth, cam)
    assert np.any(ref != 0, axis=0).sum() > 200_000


def test_normal_loss_matches_oracle():
    sc = S.surface_scene(3000, 28)
    sc.means *= 0.5
    cam = S.look_at_camera((0.0, -4.0, 2.0), (0, 0, 0.4), 45, 160, 120)
    depth, normal, _ = api.render_geometry(_gt(sc), cam)
    Np = api.pseudo_normal(depth, cam)
    loss, dN = api.normal_loss(normal, Np)
    torch.cuda.synchronize()
    Lr, gr = R.normal_loss(normal.cpu().numpy().astype(np.float64), Np.cpu().numpy().astype(np.float64))
    assert Lr > 1.0
    assert abs(float(loss.item()) - Lr) <= 1e-5 * Lr
    np.testing.assert_allclose(dN.cpu().numpy(), gr, atol=1e-6 / Lr * 10 + 1e-7, rtol=1e-5)
    # deterministic: the same bits again
    loss2, dN2 = api.normal_loss(normal, Np)
    assert torch.equal(loss, loss2) and torch.equal(dN, dN2)
    # N = N' gives zero loss and zero gradient
    l0, g0 = api.normal_loss(Np, Np)
    assert float(l0.item()) == 0.0 and torch.all(g0 == 0)


def test_normal_loss_gradient_reaches_the_splat_normals():
    """dL/dn_i through Eq. 25: the normal loss gradient fed to the render backward with the
    normals as colours, against FP64 autograd of the oracle's composite with N' held fixed."""
    sc = S.surface_scene(800, 29)
    sc.means *= 0.5
    cam = S.look_at_camera((0.0, -4.0, 2.0), (0, 0, 0.4), 45, 96, 72)
    g = _gt(sc)
    depth, normal, st = api.render_geometry(g, cam)
    Np = api.pseudo_normal(depth, cam)
    loss, dN = api.normal_loss(normal, Np)
    bg = torch.zeros(3, device="cuda")
    grads = api.render_backward(g, g.normals[None].contiguous(), cam, bg, st, dN[None].contiguous())
    d_n = grads[4][0].cpu().numpy().astype(np.float64)
    t = lambda a, rg=False: torch.tensor(np.asarray(a, np.float64), requires_grad=rg)
    nr = t(sc.normals, True)
    img = R.render(t(sc.means), t(sc.scales), t(sc.quats), t(sc.opacity), nr[None], cam)[0]
    Npd = torch.as_tensor(Np.cpu().numpy().astype(np.float64))
    m = (Npd != 0).any(0)
    L = torch.sqrt((((img - Npd) * m) ** 2).sum())
    L.backward()
    ref = nr.grad.numpy()
    assert abs(float(loss.item()) - float(L.detach())) <= 1e-4 * float(L.detach())
    scale = np.abs(ref).max()
    np.testing.assert_allclose(d_n, ref, atol=1e-4 * scale)
    assert scale > 1e-3
