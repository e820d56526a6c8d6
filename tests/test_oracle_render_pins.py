"""Pins of the FP64 splat-render oracle (Eq. 2-4) against closed forms and brute force (CPU)."""
import math

import numpy as np
import pytest
import torch

from oracle import render as R
from paper_2408_03538_gb300 import scenes as S


def _cam(w, h, f=100.0):
    return S.Camera(rot=np.eye(3, dtype=np.float32), trans=np.zeros(3, np.float32), fx=f, fy=f, cx=(w - 1) / 2,
                    cy=(h - 1) / 2, width=w, height=h, position=np.zeros(3, np.float32))


def _t(a):
    return torch.as_tensor(np.asarray(a, dtype=np.float64))


def test_single_splat_is_the_analytic_gaussian():
    cam = _cam(64, 64)
    z, s, sig = 5.0, 0.1, 0.8
    col = np.array([1.0, 0.5, 0.25])
    img = R.render(_t([[0, 0, z]]), _t([[s] * 3]), _t([[1, 0, 0, 0]]), _t([sig]), _t(col[None, None, :]), cam)
    var = (100 * s / z) ** 2 + R.DILATION
    py, px = np.mgrid[0:64, 0:64]
    d2 = (px - 31.5) ** 2 + (py - 31.5) ** 2
    a = np.minimum(0.99, sig * np.exp(-0.5 * d2 / var))
    a = np.where(a >= 1 / 255, a, 0.0)
    np.testing.assert_allclose(img[0].numpy(), col[:, None, None] * a[None], atol=1e-14)


def test_opaque_front_splat_occludes():
    cam = _cam(32, 32)
    img = R.render(_t([[0, 0, 6.0], [0, 0, 4.0]]), _t([[0.5] * 3, [0.5] * 3]), _t([[1, 0, 0, 0]] * 2),
                   _t([0.9, 0.999]), _t([[[0, 1, 0], [1, 0, 0]]]), cam)
    # pixel (15,15) is 0.5 px from both centres in x and y: the front alpha clamps to 0.99,
    # the back splat keeps 1% of its own alpha
    a_back = 0.9 * math.exp(-0.5 * 0.5 / ((100 * 0.5 / 6) ** 2 + R.DILATION))
    c = img[0, :, 15, 15].numpy()
    np.testing.assert_allclose(c, [0.99, 0.01 * a_back, 0.0], rtol=1e-12, atol=1e-15)


def _untiled(pre, opacity, colors, cam):
    """Plain per-pixel blending over every projected Gaussian in (depth, index) order."""
    H, W = cam.height, cam.width
    valid = pre["valid"].numpy()
    ids = np.nonzero(valid)[0]
    ids = ids[np.argsort(pre["depth"].detach().numpy()[ids], kind="stable")]
    m = pre["mean2d"].detach().numpy()
    con = pre["conic"].detach().numpy()
    op = opacity.numpy()
    col = colors.numpy()
    img = np.zeros((col.shape[0], 3, H, W))
    for py in range(H):
        for px in range(W):
            T = 1.0
            acc = np.zeros((col.shape[0], 3))
            for g in ids:
                dx, dy = m[g, 0] - px, m[g, 1] - py
                power = -0.5 * (con[g, 0] * dx * dx + con[g, 2] * dy * dy) - con[g, 1] * dx * dy
                if power > 0:
                    continue
                a = min(0.99, op[g] * math.exp(power))
                if a < 1 / 255:
                    continue
                if T * (1 - a) < 1e-4:
                    break
                acc += col[:, g, :] * a * T
                T *= 1 - a
            img[:, :, py, px] = acc
    return img


def test_tiled_rule_equals_untiled_brute_force_for_faint_splats():
    """With opacity <= 0.35 a splat is below 1/255 outside its 3-sigma tile rectangle, so the
    tile binning must not change any pixel (ragged 90x70 image: partial tiles on two sides)."""
    rng = np.random.default_rng(4)
    n = 120
    cam = S.look_at_camera((0, -3.5, 1.5), (0, 0, 0), 50, 90, 70)
    sc = S.isotropic_scene(n, 21)
    scales = sc.scales * 3
    op = rng.uniform(0.05, 0.35, n)
    colors = rng.uniform(0, 1, (1, n, 3))
    pre = R.preprocess(_t(sc.means), _t(scales), _t(sc.quats), cam)
    tiled = R.composite(pre, _t(op), _t(colors), cam).numpy()
    ref = _untiled(pre, _t(op), _t(colors), cam)
    np.testing.assert_allclose(tiled, ref, atol=1e-13)
    assert tiled.max() > 0.05


def test_autograd_matches_central_differences():
    rng = np.random.default_rng(7)
    n = 24
    cam = S.look_at_camera((0, -3.0, 1.0), (0, 0, 0), 50, 40, 36)
    sc = S.surface_scene(n, 5)
    means = _t(sc.means * 0.4)
    scales = _t(sc.scales * 4)
    quats = _t(sc.quats)
    op = _t(sc.opacity)
    colors = _t(rng.uniform(0, 1, (1, n, 3)))
    wimg = _t(rng.standard_normal((1, 3, 36, 40)))
    params = [means, scales, quats, op, colors]

    def loss(ps):
        return (R.render(*ps[:4], ps[4], cam) * wimg).sum()

    for p in params:
        p.requires_grad_(True)
    L = loss(params)
    grads = torch.autograd.grad(L, params)
    h = 1e-6
    checked = 0
    for pi, p in enumerate(params):
        flat = p.detach().reshape(-1)
        for k in rng.choice(flat.numel(), size=min(6, flat.numel()), replace=False):
            ps_p = [q.detach().clone() for q in params]
            ps_m = [q.detach().clone() for q in params]
            ps_p[pi].reshape(-1)[k] += h
            ps_m[pi].reshape(-1)[k] -= h
            with torch.no_grad():
                fd = (loss(ps_p) - loss(ps_m)).item() / (2 * h)
            g = grads[pi].reshape(-1)[k].item()
            assert abs(fd - g) <= 1e-5 * max(1.0, abs(fd)), (pi, k, fd, g)
            checked += 1
    assert checked >= 25
