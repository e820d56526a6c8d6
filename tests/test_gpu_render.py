"""GPU parity of relight (Eq. 14/41), the splat render (Eq. 3-4) and their backward passes
against the FP64 oracle. Images: PSNR >= 50 dB; relight: norm-wise relative error <= 1e-4;
gradients: norm-wise relative error per parameter group <= 2e-3 (FP32 atomics vs FP64)."""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import render as OR
from paper_2408_03538_gb300 import api, scenes as S

pytestmark = pytest.mark.gpu


def _cuda(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype).contiguous()


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


@pytest.mark.parametrize("order,tch,k", [(2, 1, 1), (3, 1, 5), (3, 3, 1), (3, 3, 64), (1, 1, 3), (5, 3, 7),
                                         (6, 1, 4)])
def test_relight_fp32(order, tch, k):
    rng = np.random.default_rng(order * 10 + tch + k)
    n, C = 5003, (order + 1) ** 2
    T = rng.standard_normal((n, C) if tch == 1 else (n, 3, C)).astype(np.float32)
    alb = rng.uniform(0, 1, (n, 3)).astype(np.float32)
    L = rng.standard_normal((k, 3, C)).astype(np.float32)
    col = api.relight(_cuda(T), _cuda(alb), _cuda(L), order).cpu().numpy()
    ref = oracle.relight(T, alb, L)
    err = oracle.norm_err(col.transpose(1, 0, 2), ref.transpose(1, 0, 2), 1e-6)
    assert err.max() < 1e-4


@pytest.mark.parametrize("order", [3, 5, 6])
def test_relight_glossy_fp32(order):
    """Glossy rows t_eff = M Y(v) (Eq. 41); orders 4-6 evaluate Y(v) by the Legendre recurrence."""
    rng = np.random.default_rng(3 + order)
    n, C, k = 2000, (order + 1) ** 2, 4
    T = rng.standard_normal((n, 3, C)).astype(np.float32)
    alb = rng.uniform(0, 1, (n, 3)).astype(np.float32)
    L = rng.standard_normal((k, 3, C)).astype(np.float32)
    gids = np.sort(rng.choice(n, 600, replace=False)).astype(np.int32)
    M = rng.standard_normal((600, C, C)).astype(np.float32)
    means = rng.standard_normal((n, 3)).astype(np.float32)
    cam = np.array([2.0, -5.0, 1.5], np.float32)
    col = api.relight(_cuda(T), _cuda(alb), _cuda(L), order, glossy_ids=_cuda(gids, torch.int32), M=_cuda(M),
                      means=_cuda(means), cam_pos=_cuda(cam)).cpu().numpy()
    ref = oracle.relight(T, alb, L, glossy_ids=gids, M=M, means=means, cam_pos=cam, order=order)
    err = oracle.norm_err(col.transpose(1, 0, 2), ref.transpose(1, 0, 2), 1e-6)
    assert err.max() < 1e-4


@pytest.mark.parametrize("tch,k,order", [(1, 1, 3), (3, 2, 3), (1, 9, 3), (3, 5, 4), (1, 3, 5), (3, 9, 6),
                                         (1, 4, 6)])
def test_relight_backward(tch, k, order):
    rng = np.random.default_rng(11 + k + order)
    n = 3001
    C = (order + 1) ** 2
    T = rng.standard_normal((n, C) if tch == 1 else (n, 3, C)).astype(np.float32)
    alb = rng.uniform(0, 1, (n, 3)).astype(np.float32)
    L = rng.standard_normal((k, 3, C)).astype(np.float32)
    dcol = rng.standard_normal((k, n, 3)).astype(np.float32)
    da, dT, dL = api.relight_backward(_cuda(T), _cuda(alb), _cuda(L), order, _cuda(dcol), need_dT=True)
    Tt = torch.tensor(T, dtype=torch.float64, requires_grad=True)
    At = torch.tensor(alb, dtype=torch.float64, requires_grad=True)
    Lt = torch.tensor(L, dtype=torch.float64, requires_grad=True)
    out = OR.relight_torch(Tt, At, Lt)
    out.backward(torch.tensor(dcol, dtype=torch.float64))
    assert _rel(da.cpu(), At.grad) < 1e-5
    assert _rel(dT.cpu(), Tt.grad) < 1e-5
    assert _rel(dL.cpu(), Lt.grad) < 1e-5


def _render_both(scene, colors, cam, bg=(0.0, 0.0, 0.0), tiles=None, max_pairs=None):
    g = api.GaussianTensors.from_scene(scene)
    st = api.Status()
    img, state = api.render(g, _cuda(colors), cam, _cuda(np.asarray(bg, np.float32)), max_pairs=max_pairs, status=st)
    torch.cuda.synchronize()
    assert st.read() == 0
    t = lambda a: torch.as_tensor(np.asarray(a, np.float64))
    ref = OR.render(t(scene.means), t(scene.scales), t(scene.quats), t(scene.opacity), t(colors), cam, bg, tiles=tiles)
    return img.cpu().numpy(), ref.numpy(), state


def test_render_tiny_config_psnr():
    sc = S.make_scene("tiny-1k")
    cam = S.make_camera("tiny-1k")
    rng = np.random.default_rng(2)
    colors = rng.uniform(0, 1, (1, sc.n, 3)).astype(np.float32)
    img, ref, _ = _render_both(sc, colors, cam, bg=(0.1, 0.2, 0.3))
    assert OR.psnr(img, ref, peak=1.0) >= 50.0
    assert img.std() > 0.01


def test_render_ragged_multi_light_and_culling():
    sc = S.isotropic_scene(800, 41)
    sc.means[:50, 1] = -10.0  # behind the camera plane: culled
    cam = S.look_at_camera((0, -3.5, 1.5), (0, 0, 0), 50, 97, 61)
    rng = np.random.default_rng(9)
    colors = rng.uniform(0, 1, (6, sc.n, 3)).astype(np.float32)
    img, ref, state = _render_both(sc, colors, cam)
    for l in range(6):
        assert OR.psnr(img[l], ref[l], peak=1.0) >= 50.0
    assert np.all(state.view("radius", torch.int32, (sc.n,)).cpu().numpy()[:50] == 0)


def test_render_capacity_overflow_is_reported():
    sc = S.isotropic_scene(500, 42)
    cam = S.look_at_camera((0, -3.5, 1.5), (0, 0, 0), 50, 64, 64)
    g = api.GaussianTensors.from_scene(sc)
    st = api.Status()
    colors = torch.ones((1, sc.n, 3), device="cuda")
    api.render(g, colors, cam, torch.zeros(3, device="cuda"), max_pairs=10, status=st)
    torch.cuda.synchronize()
    assert st.read() & 4


def test_render_1080p_sampled_tiles():
    """The 100k surface workload at 1920x1080: oracle on seeded sampled tiles."""
    sc = S.make_scene("surface-100k")
    cam = S.make_camera("surface-100k")
    rng = np.random.default_rng(6)
    colors = rng.uniform(0, 1, (1, sc.n, 3)).astype(np.float32)
    gx, gy = (cam.width + 15) // 16, (cam.height + 15) // 16
    tiles = [(int(rng.integers(gx)), int(rng.integers(gy))) for _ in range(24)] + [(gx - 1, gy - 1)]
    img, ref, state = _render_both(sc, colors, cam, tiles=tiles, max_pairs=8_000_000)
    for tx, ty in tiles:
        sl = (slice(None), slice(None), slice(ty * 16, min(ty * 16 + 16, cam.height)),
              slice(tx * 16, min(tx * 16 + 16, cam.width)))
        assert OR.psnr(img[sl], ref[sl], peak=1.0) >= 50.0, (tx, ty)
    assert state.n_pairs() > 100_000


def _grad_case(n=1500, W=128, H=96, k=1, seed=3):
    sc = S.surface_scene(n, seed)
    sc.means *= 0.5
    cam = S.look_at_camera((0, -4.0, 2.0), (0, 0, 0.4), 45, W, H)
    rng = np.random.default_rng(seed)
    colors = rng.uniform(0, 1, (k, sc.n, 3)).astype(np.float32)
    wimg = rng.standard_normal((k, 3, H, W)).astype(np.float32)
    return sc, cam, colors, wimg


@pytest.mark.parametrize("k", [1, 5])
def test_render_backward_matches_oracle_autograd(k):
    sc, cam, colors, wimg = _grad_case(k=k)
    g = api.GaussianTensors.from_scene(sc)
    bg = _cuda(np.array([0.05, 0.1, 0.2], np.float32))
    img, state = api.render(g, _cuda(colors), cam, bg)
    dm, ds, dq, do, dc = api.render_backward(g, _cuda(colors), cam, bg, state, _cuda(wimg))
    t = lambda a: torch.tensor(np.asarray(a, np.float64), requires_grad=True)
    ps = [t(sc.means), t(sc.scales), t(sc.quats), t(sc.opacity), t(colors)]
    ref = OR.render(*ps[:4], ps[4], cam, bg=(0.05, 0.1, 0.2))
    (ref * torch.tensor(wimg, dtype=torch.float64)).sum().backward()
    for got, p, name in zip((dm, ds, dq, do, dc), ps, ("means", "scales", "quats", "opacity", "colors")):
        assert _rel(got.cpu(), p.grad) < 2e-3, name
    assert OR.psnr(img.cpu().numpy(), ref.detach().numpy(), peak=1.0) >= 50


def test_relit_render_autograd_end_to_end():
    """d(L2 loss)/d(light SH, albedo, geometry) through relight + render on the GPU equals
    the oracle's FP64 autograd gradient (2k-Gaussian anisotropic subset; rotation included)."""
    sc, cam, _, _ = _grad_case(n=2000, W=120, H=90, seed=8)
    order = 3
    rng = np.random.default_rng(1)
    T = (rng.standard_normal((sc.n, 3, 16)) * 0.3 + np.eye(16)[0] * 1.5).astype(np.float32)
    Lsh = S.env_lights(1, order, 5)
    target = rng.uniform(0, 0.5, (1, 3, cam.height, cam.width)).astype(np.float32)
    g = api.GaussianTensors.from_scene(sc)
    leaves = [g.means.clone().requires_grad_(), g.scales.clone().requires_grad_(), g.quats.clone().requires_grad_(),
              g.opacity.clone().requires_grad_(), g.albedo.clone().requires_grad_(),
              _cuda(Lsh).requires_grad_()]
    img = api.relit_render(*leaves, _cuda(T), g.normals, cam, order)
    loss, dimg = api.l2_loss(img.detach().contiguous(), _cuda(target))
    img.backward(dimg)
    t = lambda a: torch.tensor(np.asarray(a, np.float64), requires_grad=True)
    ps = [t(sc.means), t(sc.scales), t(sc.quats), t(sc.opacity), t(sc.albedo), t(Lsh)]
    col = OR.relight_torch(torch.tensor(T, dtype=torch.float64), ps[4], ps[5])
    ref = OR.render(*ps[:4], col, cam)
    rl = ((ref - torch.tensor(target, dtype=torch.float64)) ** 2).mean()
    rl.backward()
    assert abs(loss.item() - rl.item()) <= 1e-4 * rl.item()
    for got, p, name in zip(leaves, ps, ("means", "scales", "quats", "opacity", "albedo", "light")):
        assert _rel(got.grad.cpu(), p.grad) < 2e-3, name


@pytest.mark.parametrize("order,k,n,tch", [(3, 1, 5003, 1), (3, 64, 20000, 1), (2, 4, 129, 1), (1, 2, 128, 1),
                                           (3, 85, 777, 1), (3, 64, 20000, 3), (2, 5, 777, 3), (1, 1, 129, 3),
                                           (3, 160, 3001, 3), (3, 10, 4099, 1),
                                           (4, 8, 3001, 3), (4, 85, 1025, 1), (5, 64, 2049, 1), (5, 80, 999, 3),
                                           (6, 64, 5003, 3), (6, 85, 777, 1), (6, 1, 129, 1), (6, 13, 20000, 3)])
def test_relight_tensor_core_bf16x3(order, k, n, tch):
    """tcgen05 relight with the 3-term BF16 split meets the FP32 bar (1e-4 norm-wise), for
    scalar and RGB transfer, ragged row tails and light counts that are not multiples of 8."""
    rng = np.random.default_rng(order * 100 + k + tch)
    C = (order + 1) ** 2
    T = rng.standard_normal((n, C) if tch == 1 else (n, 3, C)).astype(np.float32)
    alb = rng.uniform(0, 1, (n, 3)).astype(np.float32)
    L = rng.standard_normal((k, 3, C)).astype(np.float32)
    col = api.relight(_cuda(T), _cuda(alb), _cuda(L), order, precision=1).cpu().numpy()
    ref = oracle.relight(T, alb, L)
    err = oracle.norm_err(col.transpose(1, 0, 2), ref.transpose(1, 0, 2), 1e-3)
    assert np.all(np.isfinite(col))
    assert err.max() < 1e-4, err.max()


def test_relight_tensor_core_plain_bf16_error_is_bf16_sized():
    rng = np.random.default_rng(7)
    n, C, k = 4096, 16, 8
    T = rng.standard_normal((n, C)).astype(np.float32)
    alb = rng.uniform(0, 1, (n, 3)).astype(np.float32)
    L = rng.standard_normal((k, 3, C)).astype(np.float32)
    col = api.relight(_cuda(T), _cuda(alb), _cuda(L), 3, precision=2).cpu().numpy()
    ref = oracle.relight(T, alb, L)
    err = oracle.norm_err(col.transpose(1, 0, 2), ref.transpose(1, 0, 2), 1e-3)
    assert 1e-5 < np.median(err) < 2e-2  # plain BF16 operands: about 2^-8 relative


@pytest.mark.parametrize("order,k", [(3, 64), (6, 32)])
def test_relight_tensor_core_with_glossy_rows(order, k):
    """BF16x3 tensor cores for every row, then the glossy rows rewritten in FP32 (Eq. 41)."""
    rng = np.random.default_rng(17 + order)
    n, C = 6000, (order + 1) ** 2
    T = rng.standard_normal((n, 3, C)).astype(np.float32)
    alb = rng.uniform(0, 1, (n, 3)).astype(np.float32)
    L = rng.standard_normal((k, 3, C)).astype(np.float32)
    gids = np.sort(rng.choice(n, size=1800, replace=False)).astype(np.int32)
    M = rng.standard_normal((gids.size, C, C)).astype(np.float32) * 0.2
    means = rng.uniform(-1, 1, (n, 3)).astype(np.float32)
    cam = np.array([0.5, -3.0, 1.0], np.float32)
    col = api.relight(_cuda(T), _cuda(alb), _cuda(L), order, precision=1, glossy_ids=_cuda(gids, torch.int32),
                      M=_cuda(M), means=_cuda(means), cam_pos=_cuda(cam)).cpu().numpy()
    ref = oracle.relight(T, alb, L, glossy_ids=gids, M=M, means=means, cam_pos=cam, order=order)
    err = oracle.norm_err(col.transpose(1, 0, 2), ref.transpose(1, 0, 2), 1e-3)
    assert err.max() < 1e-4, err.max()


def test_relight_tensor_core_rejects_unsupported():
    with pytest.raises(Exception):  # 3k > 256 output columns for scalar transfer
        api.relight(torch.zeros((10, 16), device="cuda"), torch.zeros((10, 3), device="cuda"),
                    torch.zeros((90, 3, 16), device="cuda"), 3, precision=1)
    with pytest.raises(Exception):  # more lights than one launch holds
        api.relight(torch.zeros((10, 3, 16), device="cuda"), torch.zeros((10, 3), device="cuda"),
                    torch.zeros((300, 3, 16), device="cuda"), 3, precision=1)
    with pytest.raises(Exception):  # order 6, RGB transfer: the lights of four K blocks exceed shared memory
        api.relight(torch.zeros((10, 3, 49), device="cuda"), torch.zeros((10, 3), device="cuda"),
                    torch.zeros((65, 3, 49), device="cuda"), 6, precision=1)


def test_relit_render_through_transfer_end_to_end():
    """The whole differentiable path: P = shadowed transfer of the Gaussians, colours =
    relight(P), image = render. d(L2 loss)/d(geometry, normals, albedo, light) against FP64
    autograd through the brute-force transfer, relight and render (600 crowded surface
    Gaussians, order 3, S = 48): the geometry gradient is the sum of the rasterizer's and the
    transfer's."""
    from oracle import transfer_torch as TT

    sc = S.surface_scene(600, 12)
    sc.means *= 0.4
    sc.scales *= 1.5
    cam = S.look_at_camera((0, -4.0, 2.0), (0, 0, 0.2), 40, 96, 80)
    order = 3
    dirs = S.direction_set(48, 7)
    rng = np.random.default_rng(2)
    Lsh = S.env_lights(1, order, 4)
    target = rng.uniform(0, 0.5, (1, 3, cam.height, cam.width)).astype(np.float32)
    g = api.GaussianTensors.from_scene(sc)
    names = ("means", "scales", "quats", "opacity", "albedo", "light", "normals")
    leaves = [g.means.clone().requires_grad_(), g.scales.clone().requires_grad_(), g.quats.clone().requires_grad_(),
              g.opacity.clone().requires_grad_(), g.albedo.clone().requires_grad_(), _cuda(Lsh).requires_grad_(),
              g.normals.clone().requires_grad_()]
    P = api.shadowed_transfer(leaves[0], leaves[1], leaves[2], leaves[3], leaves[6], g.albedo, _cuda(dirs), order,
                              t_min=0.0)
    img = api.relit_render(*leaves[:6], P, g.normals, cam, order)
    loss, dimg = api.l2_loss(img.detach().contiguous(), _cuda(target))
    img.backward(dimg)
    t = lambda a: torch.tensor(np.asarray(a, np.float64), requires_grad=True)
    ps = [t(sc.means), t(sc.scales), t(sc.quats), t(sc.opacity), t(sc.albedo), t(Lsh), t(sc.normals)]
    Pr = TT.transfer_P(ps[0], ps[1], ps[2], ps[3], ps[6], dirs, oracle.sh(order, dirs))
    ref = OR.render(*ps[:4], OR.relight_torch(Pr, ps[4], ps[5]), cam)
    rl = ((ref - torch.tensor(target, dtype=torch.float64)) ** 2).mean()
    rl.backward()
    assert abs(loss.item() - rl.item()) <= 1e-4 * rl.item()
    for got, p, name in zip(leaves, ps, names):
        assert _rel(got.grad.cpu(), p.grad) < 2e-3, name
    assert float(ps[6].grad.abs().sum()) > 0  # the normals get their gradient from the transfer only


def test_diff_300k_central_differences_on_64_parameters():
    """300,000 isotropic Gaussians, order 3, relit 1080p image with an L2 loss against a seeded
    target: the hand-written gradient against central differences (h = 1e-3) of the GPU
    forward on 64 seeded parameters (16 light coefficients; 48 albedo, opacity, mean, scale
    and rotation entries of Gaussians that reach the image; the camera looks along y, z). T is the precomputed transfer,
    a constant as in the paper's optimisation."""
    sc = S.make_scene("diff-300k")
    cam = S.make_camera("diff-300k")
    order = 3
    g = api.GaussianTensors.from_scene(sc)
    bvh = api.build_bvh(g)
    dirs = _cuda(S.direction_set(128, S.config_seed(3)))
    T = api.precompute_transfer(g, bvh, dirs, order)["P"]
    Lsh = _cuda(S.env_lights(1, order, S.config_seed(3)))
    rng = np.random.default_rng(64)
    target = _cuda(rng.uniform(0, 0.5, (1, 3, cam.height, cam.width)).astype(np.float32))
    base = [g.means, g.scales, g.quats, g.opacity, g.albedo, Lsh]
    leaves = [b.clone().requires_grad_() for b in base]
    img = api.relit_render(*leaves, T, g.normals, cam, order, max_pairs=40_000_000)
    loss, dimg = api.l2_loss(img.detach().contiguous(), target)
    img.backward(dimg)
    grads = [l.grad.detach() for l in leaves]
    tgt64 = target.double()

    def L(vals):
        with torch.no_grad():
            im = api.relit_render(*vals, T, g.normals, cam, order, max_pairs=40_000_000)
            return ((im.double() - tgt64) ** 2).mean()

    visible = torch.nonzero(grads[4].abs().sum(1) > 0).flatten().cpu().numpy()
    picks = [(5, (0, int(c), int(k))) for c, k in zip(rng.integers(0, 3, 16), rng.integers(0, 16, 16))]
    # (field, entries per Gaussian, how many): albedo, opacity, means (x only), scales, quats.
    # The camera's right axis is world x, so moving a mean along x leaves every depth as it was;
    # along y or z a 1e-3 step can swap two overlapping Gaussians in the front-to-back order,
    # a jump of the image that no gradient of the 3DGS composite sees.
    for field, width, count in ((4, 3, 10), (3, 1, 10), (0, 1, 10), (1, 3, 9), (2, 4, 9)):
        for _ in range(count):
            i = int(rng.choice(visible))
            picks.append((field, (i, 0) if field == 0 else (i,) if width == 1 else (i, int(rng.integers(width)))))
    assert len(picks) == 64
    h = 1e-3
    bad = []
    scale = {f: float(grads[f].abs().max()) for f in range(6)}
    # the rotation of an isotropic Gaussian changes nothing: both sides are FP32 noise, held
    # against the scale of the other geometry gradients
    scale[2] = max(scale[0], scale[1])
    for field, ix in picks:
        vp = [b.clone() for b in base]
        vm = [b.clone() for b in base]
        vp[field][ix] += h
        vm[field][ix] -= h
        fd = float(L(vp) - L(vm)) / (2 * h)
        gv = float(grads[field][ix])
        if abs(fd - gv) > 2e-2 * abs(fd) + 1e-3 * scale[field]:
            bad.append((field, ix, fd, gv))
    assert not bad, bad[:8]


def test_relight_1m_64_lights_tensor_cores_full_size():
    """The 1M-splat, 64-light relight of the tiled glossy workload on the tensor cores (BF16x3,
    RGB transfer, 30 % glossy rows rewritten in FP32): sampled rows against the oracle."""
    rng = np.random.default_rng(64)
    n, C, k = 1_000_000, 16, 64
    T = (rng.standard_normal((n, 3, C)) * 0.3).astype(np.float32)
    T[:, :, 0] += 1.5
    alb = rng.uniform(0, 1, (n, 3)).astype(np.float32)
    L = S.env_lights(k, 3, 99)
    gids = np.nonzero(rng.random(n) < 0.3)[0].astype(np.int32)
    M = (rng.standard_normal((gids.size, C, C)) * 0.1).astype(np.float32)
    means = rng.uniform(-20, 20, (n, 3)).astype(np.float32)
    cam = np.array([0.0, -40.0, 14.0], np.float32)
    col = api.relight(_cuda(T), _cuda(alb), _cuda(L), 3, precision=1, glossy_ids=_cuda(gids, torch.int32),
                      M=_cuda(M), means=_cuda(means), cam_pos=_cuda(cam))
    rows = np.sort(rng.choice(n, 4096, replace=False))
    got = col[:, torch.from_numpy(rows).cuda(), :].cpu().numpy()
    gsel = np.isin(gids, rows)
    ref = oracle.relight(T[rows], alb[rows], L, glossy_ids=np.searchsorted(rows, gids[gsel]), M=M[gsel],
                         means=means[rows], cam_pos=cam, order=3)
    err = oracle.norm_err(got.transpose(1, 0, 2), ref.transpose(1, 0, 2), 1e-3)
    assert gsel.sum() > 1000
    assert err.max() < 1e-4, err.max()


# ---- pixel-space relight of many lights ----------------------------------------------------
@pytest.mark.parametrize("precision,bar,order,tch", [(0, 50.0, 3, 3), (1, 50.0, 3, 3), (2, 30.0, 3, 3),
                                                     (1, 50.0, 2, 1), (0, 50.0, 1, 3), (1, 50.0, 1, 1),
                                                     (0, 50.0, 6, 3), (1, 50.0, 6, 3), (1, 50.0, 5, 1),
                                                     (0, 50.0, 4, 1)])
def test_render_relit_matches_oracle(precision, bar, order, tch):
    """Composite the splats' (rho/pi) T once, contract per pixel with 12 lights: equals the FP64
    oracle's relight + composite of each light (30 % glossy splats, background; RGB or scalar
    transfer, SH orders 1-6)."""
    sc = S.surface_scene(1500, 44)
    sc.means *= 0.5
    rng = np.random.default_rng(44)
    n, C, k = sc.n, (order + 1) ** 2, 12
    T = (rng.standard_normal((n, 3, C) if tch == 3 else (n, C)) * 0.3).astype(np.float32)
    T[..., 0] += 1.2
    L = S.env_lights(k, order, 45)
    gids = np.sort(rng.choice(n, 450, replace=False)).astype(np.int32)
    M = (rng.standard_normal((gids.size, C, C)) * 0.1 + np.eye(C) * 0.8).astype(np.float32)
    cam = S.look_at_camera((0, -4.0, 2.0), (0, 0, 0.4), 45, 96, 80)
    bg = np.array([0.05, 0.1, 0.2], np.float32)
    g = api.GaussianTensors.from_scene(sc)
    st = api.Status()
    img, _ = api.render_relit(g, _cuda(T), _cuda(L), cam, order, bg=_cuda(bg), precision=precision,
                              glossy_ids=_cuda(gids, torch.int32), M=_cuda(M), status=st)
    torch.cuda.synchronize()
    assert st.read() == 0
    col = oracle.relight(T, sc.albedo, L, glossy_ids=gids, M=M, means=sc.means, cam_pos=np.asarray(cam.position),
                         order=order)
    t = lambda a: torch.as_tensor(np.asarray(a, np.float64))
    ref = OR.render(t(sc.means), t(sc.scales), t(sc.quats), t(sc.opacity), t(col), cam, tuple(bg)).numpy()
    img = img.cpu().numpy()
    peak = float(np.abs(ref).max())
    for l in range(k):
        assert OR.psnr(img[l], ref[l], peak=peak) >= bar, l
    assert img.std() > 1e-3


def test_render_relit_full_size_64_lights_equals_per_light_path():
    """1M tiled glossy splats, 64 lights, 1920x1080: the pixel-space relight (tcgen05 BF16x3)
    equals relight + 64 composites (FP32) to >= 50 dB on every light, and is timed beside it;
    on seeded sampled tiles it matches the FP64 oracle's relight + composite (six lights)."""
    sc = S.make_scene("tiled-1m-glossy")
    cam = S.make_camera("tiled-1m-glossy")
    rng = np.random.default_rng(8)
    n, C, k = sc.n, 16, 64
    T = torch.from_numpy((rng.standard_normal((n, 3, C)) * 0.3 + np.eye(C)[0] * 1.2).astype(np.float32)).cuda()
    L = _cuda(S.env_lights(k, 3, 9))
    gids = torch.from_numpy(np.nonzero(sc.glossy_mask)[0].astype(np.int32)).cuda()
    M = torch.from_numpy((rng.standard_normal((gids.numel(), C, C)) * 0.1 + np.eye(C) * 0.8)
                         .astype(np.float32)).cuda()
    g = api.GaussianTensors.from_scene(sc)
    bg = _cuda(np.array([0.05, 0.1, 0.2], np.float32))
    cam_pos = _cuda(np.asarray(cam.position, np.float32))
    st = api.Status()
    state = api.RenderState(n, cam.width, cam.height, 40_000_000)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    img_px, _ = api.render_relit(g, T, L, cam, 3, bg=bg, precision=1, glossy_ids=gids, M=M, state=state, status=st)
    ev[0].record()
    img_px, _ = api.render_relit(g, T, L, cam, 3, bg=bg, precision=1, glossy_ids=gids, M=M, state=state, status=st,
                                 out=img_px)
    ev[1].record()
    col = api.relight(T, g.albedo, L, 3, glossy_ids=gids, M=M, means=g.means, cam_pos=cam_pos)
    img_pl, _ = api.render(g, col, cam, bg, state=state, status=st)
    ev[2].record()
    torch.cuda.synchronize()
    assert st.read() == 0
    ms_px, ms_pl = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
    print(f"pixel-space {ms_px:.2f} ms, per-light {ms_pl:.2f} ms")
    a, b = img_px.double(), img_pl.double()
    peak = float(b.abs().max())
    for l in range(k):
        mse = float(((a[l] - b[l]) ** 2).mean())
        assert mse == 0 or 10 * math.log10(peak * peak / mse) >= 50.0, l
    # the FP64 oracle on seeded sampled tiles, for lights spread over the 64
    sel = [0, 9, 21, 33, 47, 63]
    ref_col = oracle.relight(T.cpu().numpy(), sc.albedo, L.cpu().numpy()[sel], glossy_ids=gids.cpu().numpy(),
                             M=M.cpu().numpy(), means=sc.means, cam_pos=np.asarray(cam.position), order=3)
    gx, gy = (cam.width + 15) // 16, (cam.height + 15) // 16
    trng = np.random.default_rng(81)
    tiles = [(int(trng.integers(gx // 4, 3 * gx // 4)), int(trng.integers(gy // 4, 3 * gy // 4))) for _ in range(12)]
    t = lambda v: torch.as_tensor(np.asarray(v, np.float64))
    ref = OR.render(t(sc.means), t(sc.scales), t(sc.quats), t(sc.opacity), t(ref_col), cam,
                    tuple(bg.cpu().numpy().tolist()), tiles=tiles).numpy()
    got = img_px.cpu().numpy()[sel]
    sls = [(slice(None), slice(None), slice(ty * 16, ty * 16 + 16), slice(tx * 16, tx * 16 + 16)) for tx, ty in tiles]
    peak = max(float(np.abs(ref[sl]).max()) for sl in sls)
    for (tx, ty), sl in zip(tiles, sls):
        assert OR.psnr(got[sl], ref[sl], peak=peak) >= 50.0, (tx, ty)
    assert sum(float(ref[sl].std()) > 1e-3 for sl in sls) >= 6  # the sample sees the scene


def test_depth_and_normal_maps_match_oracle():
    """Eq. 23 and Eq. 25: composites of each splat's view-space depth and normal (background 0)
    against the FP64 oracle's composite of the same per-splat values."""
    sc = S.surface_scene(2000, 51)
    sc.means *= 0.5
    cam = S.look_at_camera((0, -4.0, 2.0), (0, 0, 0.4), 45, 120, 90)
    g = api.GaussianTensors.from_scene(sc)
    st = api.Status()
    depth, normal, _ = api.render_geometry(g, cam, status=st)
    torch.cuda.synchronize()
    assert st.read() == 0
    m = np.asarray(sc.means, np.float64)
    d = m @ np.asarray(cam.rot, np.float64)[2] + float(np.asarray(cam.trans, np.float64)[2])
    feats = np.zeros((2, sc.n, 3))
    feats[0, :, 0] = d
    feats[1] = np.asarray(sc.normals, np.float64)
    t = lambda a: torch.as_tensor(np.asarray(a, np.float64))
    ref = OR.render(t(sc.means), t(sc.scales), t(sc.quats), t(sc.opacity), t(feats), cam).numpy()
    dref, nref = ref[0, 0], ref[1]
    assert OR.psnr(depth.cpu().numpy(), dref, peak=float(np.abs(dref).max())) >= 60.0
    assert OR.psnr(normal.cpu().numpy(), nref, peak=1.0) >= 60.0
    assert float(dref.max()) > 1.0 and float(np.abs(nref).max()) > 0.5
