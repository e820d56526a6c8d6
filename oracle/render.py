"""FP64 PyTorch splat renderer -- TEST INFRASTRUCTURE ONLY (part of the PRTGS oracle).

Restates the 3D Gaussian splatting image formation the paper builds on (Sec. 3.1):
covariance from rotation and scale (Eq. 2), EWA projection Sigma' = J W Sigma W^T J^T
(Eq. 3) and front-to-back alpha blending C = sum_i c_i a_i prod_{j<i} (1 - a_j) (Eq. 4).

The paper gives only those equations; the remaining rules are the 3DGS rasteriser's
(Kerbl et al. 2023, the paper's [3dgs]), taken as the reading of Eq. 3-4:
  * cull when the camera-space depth z <= near (0.2);
  * Jacobian evaluated with x/z, y/z clamped to 1.3 x the half field of view;
  * 0.3 px^2 added to the diagonal of Sigma'; conic = inverse of Sigma';
  * radius = ceil(3 sqrt(lambda_max)), lambda from the 2x2 eigenvalues with the
    discriminant floored at 0.1;
  * 16x16-pixel tiles; a Gaussian is binned to tiles x in [floor((mx-r)/16), floor((mx+r)/16)]
    (likewise y), clipped to the grid; pixels only see Gaussians binned to their tile;
  * per pixel, Gaussians in (depth, index) order; power = -0.5 (a dx^2 + c dy^2) - b dx dy
    with d = mean2d - pixel centre; skip power > 0; alpha = min(0.99, sigma e^power);
    skip alpha < 1/255; stop before a Gaussian that would take T below 1e-4;
    the background is added with the final transmittance.

Everything is differentiable through autograd with the discrete decisions frozen, which
gives the oracle's gradients.
"""
from __future__ import annotations

import math

import numpy as np
import torch

TILE = 16
NEAR = 0.2
ALPHA_MAX = 0.99
ALPHA_MIN = 1.0 / 255.0
T_STOP = 1e-4
DILATION = 0.3


def _t(a, requires_grad=False):
    t = torch.as_tensor(np.asarray(a), dtype=torch.float64).clone()
    if requires_grad:
        t.requires_grad_(True)
    return t


def quat_to_rot(q):
    q = q / torch.linalg.norm(q, dim=1, keepdim=True)
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    return torch.stack([
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        torch.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        torch.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], dim=1)


def preprocess(means, scales, quats, cam):
    """Projection of every Gaussian (Eq. 2-3). Returns a dict of FP64 tensors."""
    Rw = torch.as_tensor(np.asarray(cam.rot, dtype=np.float64))
    tw = torch.as_tensor(np.asarray(cam.trans, dtype=np.float64))
    fx, fy, cx, cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    W, H = int(cam.width), int(cam.height)
    R = quat_to_rot(quats)
    Sig = R @ torch.diag_embed(scales * scales) @ R.transpose(1, 2)
    p = means @ Rw.T + tw
    x, y, z = p[:, 0], p[:, 1], p[:, 2]
    valid = (z > NEAR).detach()
    zs = torch.where(valid, z, torch.ones_like(z))
    limx = 1.3 * (0.5 * W / fx)
    limy = 1.3 * (0.5 * H / fy)
    tx = torch.clamp(x / zs, -limx, limx) * zs
    ty = torch.clamp(y / zs, -limy, limy) * zs
    zero = torch.zeros_like(zs)
    J = torch.stack([torch.stack([fx / zs, zero, -fx * tx / (zs * zs)], -1),
                     torch.stack([zero, fy / zs, -fy * ty / (zs * zs)], -1)], dim=1)  # [N,2,3]
    Mt = J @ Rw.unsqueeze(0)
    cov = Mt @ Sig @ Mt.transpose(1, 2)
    a = cov[:, 0, 0] + DILATION
    b = cov[:, 0, 1]
    c = cov[:, 1, 1] + DILATION
    det = a * c - b * b
    valid = valid & (det > 0).detach()
    dets = torch.where(valid, det, torch.ones_like(det))
    conic = torch.stack([c / dets, -b / dets, a / dets], -1)
    mid = 0.5 * (a + c)
    disc = torch.sqrt(torch.clamp(mid * mid - det, min=0.1))
    lam = torch.maximum(mid + disc, mid - disc)
    radius = torch.ceil(3.0 * torch.sqrt(lam.detach()))
    mean2d = torch.stack([fx * x / zs + cx, fy * y / zs + cy], -1)
    gx, gy = (W + TILE - 1) // TILE, (H + TILE - 1) // TILE
    m2 = mean2d.detach()
    xmin = torch.clamp(torch.floor((m2[:, 0] - radius) / TILE), 0, gx)
    xmax = torch.clamp(torch.floor((m2[:, 0] + radius) / TILE) + 1, 0, gx)
    ymin = torch.clamp(torch.floor((m2[:, 1] - radius) / TILE), 0, gy)
    ymax = torch.clamp(torch.floor((m2[:, 1] + radius) / TILE) + 1, 0, gy)
    valid = valid & (radius > 0) & (xmax > xmin) & (ymax > ymin)
    return dict(mean2d=mean2d, conic=conic, depth=z, radius=radius, valid=valid,
                rect=torch.stack([xmin, ymin, xmax, ymax], -1).long(), grid=(gx, gy))


def composite(pre, opacity, colors, cam, bg=(0.0, 0.0, 0.0), tiles=None, return_T=False):
    """Front-to-back blending (Eq. 4) tile by tile. colors [k,N,3] -> image [k,3,H,W].

    ``tiles``: optional list of (tx,ty) to render (others stay zero), for sampled checks.
    """
    W, H = int(cam.width), int(cam.height)
    gx, gy = pre["grid"]
    k = colors.shape[0]
    img = torch.zeros((k, 3, H, W), dtype=torch.float64)
    Tfin = torch.ones((H, W), dtype=torch.float64)
    bg = torch.as_tensor(bg, dtype=torch.float64)
    valid = pre["valid"]
    rect = pre["rect"]
    depth = pre["depth"].detach()
    ids_all = torch.nonzero(valid).flatten()
    # depth order with ties broken by index (stable sort on depth of index-ordered ids)
    order = ids_all[torch.sort(depth[ids_all], stable=True).indices]
    r = rect[order]
    if tiles is None:
        tiles = [(tx, ty) for ty in range(gy) for tx in range(gx)]
    out_rows = []
    for tx, ty in tiles:
        sel = (r[:, 0] <= tx) & (tx < r[:, 2]) & (r[:, 1] <= ty) & (ty < r[:, 3])
        g = order[sel]
        x0, y0 = tx * TILE, ty * TILE
        xs = torch.arange(x0, min(x0 + TILE, W), dtype=torch.float64)
        ys = torch.arange(y0, min(y0 + TILE, H), dtype=torch.float64)
        py, px = torch.meshgrid(ys, xs, indexing="ij")
        pix = torch.stack([px.flatten(), py.flatten()], -1)  # [P,2]
        if g.numel() == 0:
            out = bg[None, :, None].expand(k, 3, pix.shape[0])
            Tt = torch.ones(pix.shape[0], dtype=torch.float64)
        else:
            m = pre["mean2d"][g]
            con = pre["conic"][g]
            d = m[None, :, :] - pix[:, None, :]  # [P,G,2]
            power = -0.5 * (con[None, :, 0] * d[..., 0] ** 2 + con[None, :, 2] * d[..., 1] ** 2) \
                - con[None, :, 1] * d[..., 0] * d[..., 1]
            alpha = torch.clamp(opacity[g][None, :] * torch.exp(power), max=ALPHA_MAX)
            keep = ((power <= 0) & (alpha >= ALPHA_MIN)).detach()
            a = torch.where(keep, alpha, torch.zeros_like(alpha))
            one_m = 1.0 - a
            cp = torch.cumprod(one_m, dim=1)
            Tex = torch.cat([torch.ones_like(cp[:, :1]), cp[:, :-1]], dim=1)
            incl = (keep & (Tex * one_m >= T_STOP)).detach()
            wgt = torch.where(incl, a * Tex, torch.zeros_like(a))  # [P,G]
            Tt = torch.prod(torch.where(incl, one_m, torch.ones_like(one_m)), dim=1)
            out = torch.einsum("pg,kgc->kcp", wgt, colors[:, g, :]) + Tt[None, None, :] * bg[None, :, None]
        out_rows.append((x0, y0, len(xs), len(ys), out, Tt))
    # assemble without in-place ops on a graph leaf
    rows = []
    for x0, y0, nx, ny, out, Tt in out_rows:
        rows.append((x0, y0, nx, ny, out.reshape(k, 3, ny, nx), Tt.reshape(ny, nx)))
    img_parts = img.clone()
    for x0, y0, nx, ny, o, Tt in rows:
        img_parts = img_parts.index_put((torch.arange(k)[:, None, None, None], torch.arange(3)[None, :, None, None],
                                         torch.arange(y0, y0 + ny)[None, None, :, None],
                                         torch.arange(x0, x0 + nx)[None, None, None, :]), o)
        Tfin[y0:y0 + ny, x0:x0 + nx] = Tt.detach()
    return (img_parts, Tfin) if return_T else img_parts


def render(means, scales, quats, opacity, colors, cam, bg=(0.0, 0.0, 0.0), tiles=None, return_T=False):
    """Full render: preprocess (Eq. 2-3) then composite (Eq. 4). All tensors FP64."""
    pre = preprocess(means, scales, quats, cam)
    return composite(pre, opacity, colors, cam, bg, tiles, return_T)


def relight_torch(T, albedo, L):
    """colors[k,N,3] = (rho/pi) (T . L_k) (Eq. 14), T [N,C] or [N,3,C]."""
    if T.dim() == 2:
        dot = torch.einsum("nc,khc->knh", T, L)
    else:
        dot = torch.einsum("nhc,khc->knh", T, L)
    return dot * (albedo / math.pi)[None]


def psnr(a, b, peak=None):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    mse = np.mean((a - b) ** 2)
    if peak is None:
        peak = max(float(np.max(np.abs(b))), 1e-12)
    return float("inf") if mse == 0 else 10.0 * math.log10(peak * peak / mse)


# ------------------------------------------------------------------------------------------
# Pseudo-normal from the depth map and the normal loss (Sec. 4.3, Eq. 23-25)
# ------------------------------------------------------------------------------------------
def backproject(depth, cam):
    """World-space points X[H,W,3] of a view-space depth map: the pixel (u, v) (centre at
    integer coordinates, the projection u = fx x/z + cx of ``preprocess``) at depth z is the
    camera-space point z ((u - cx)/fx, (v - cy)/fy, 1), taken to the world by R^T (x - t)."""
    D = np.asarray(depth, dtype=np.float64)
    H, W = D.shape
    R = np.asarray(cam.rot, dtype=np.float64)
    t = np.asarray(cam.trans, dtype=np.float64)
    u = (np.arange(W, dtype=np.float64) - float(cam.cx)) / float(cam.fx)
    v = (np.arange(H, dtype=np.float64) - float(cam.cy)) / float(cam.fy)
    Xc = np.stack([D * u[None, :], D * v[:, None], D], axis=-1)
    return (Xc - t) @ R


def pseudo_normal(depth, cam):
    """Pseudo-normal map N'[3,H,W] of a depth map (Eq. 24: "computed from D").

    Reading: the paper does not say how. As in the works it cites for it, each pixel is
    back-projected to its 3D point (``backproject``) and N' is the unit normal of the surface
    those points span, from central differences: N' ~ (X(u,v+1) - X(u,v-1)) x (X(u+1,v) -
    X(u-1,v)), the orientation that faces the camera, in world space. It is defined where the
    pixel and its four neighbours all have depth > 0 (the composite of Eq. 23 is 0 where no
    splat contributes) and the pixel is not on the image border; elsewhere N' = 0.
    """
    D = np.asarray(depth, dtype=np.float64)
    H, W = D.shape
    X = backproject(D, cam)
    N = np.zeros((3, H, W))
    if H < 3 or W < 3:
        return N
    du = X[1:-1, 2:] - X[1:-1, :-2]
    dv = X[2:, 1:-1] - X[:-2, 1:-1]
    n = np.cross(dv, du)
    ln = np.linalg.norm(n, axis=-1)
    ok = ((D[1:-1, 1:-1] > 0) & (D[1:-1, 2:] > 0) & (D[1:-1, :-2] > 0) & (D[2:, 1:-1] > 0) & (D[:-2, 1:-1] > 0)
          & (ln > 0))
    n = np.where(ok[..., None], n / np.where(ln > 0, ln, 1.0)[..., None], 0.0)
    N[:, 1:-1, 1:-1] = np.moveaxis(n, -1, 0)
    return N


def normal_loss(normal, pseudo):
    """L_normal = ||N - N'|| (Eq. 25) and dL/dN.

    Reading: ||.|| is the Euclidean (Frobenius) norm of the difference of the two maps, taken
    over the pixels where N' is defined (N' != 0); N' is the guide and carries no gradient
    (it serves as guidance for the splats' normals). dL/dN = (N - N') / L on those pixels,
    0 elsewhere and when L = 0.
    """
    N = np.asarray(normal, dtype=np.float64)
    Np = np.asarray(pseudo, dtype=np.float64)
    m = np.any(Np != 0, axis=0)
    diff = np.where(m[None], N - Np, 0.0)
    L = float(np.sqrt(np.sum(diff * diff)))
    return L, (diff / L if L > 0 else np.zeros_like(diff))
