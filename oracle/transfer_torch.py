"""FP64 PyTorch restatement of the shadowed transfer P and of the bounces -- TEST INFRASTRUCTURE ONLY.

Differentiable counterpart of oracle_trace's P (Eq. 29 projected by Eq. 9, visibility from
Eq. 27 read as the Gaussian's maximum along the ray, Eq. 4 along a ray), for the gradients of
the transfer with respect to the Gaussians: brute force over every (receiver, occluder,
direction) triple, so only small scenes. The hit set (t* > 0, D^2 <= 9) and the hemisphere
test (n.w > 0) are decided on detached values and frozen; the visibility product, the opacity
terms, the cosine and the ray origin carry the gradient.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from .render import quat_to_rot


def _hit_test(means, Sinv, recv_means, d, j0, j1):
    """Frozen hit set of the receivers' rays against Gaussians j0..j1: [Ni,Nj,S] booleans
    (t* > 0 and D^2 <= 9, the closest approach in Sigma^-1)."""
    u = recv_means[:, None, :] - means[None, j0:j1, :]  # o - mu_j
    Sd = torch.einsum("jab,sb->jsa", Sinv[j0:j1], d)
    a = torch.einsum("sa,jsa->js", d, Sd)
    b = torch.einsum("ija,jsa->ijs", u, Sd)
    cc = torch.einsum("ija,jab,ijb->ij", u, Sinv[j0:j1], u)
    t = -b / a[None]
    D2 = cc[:, :, None] - b * b / a[None]
    return (t > 0) & (D2 <= 9.0)


def transfer_P(means, scales, quats, opacity, normals, dirs, Y, recv=None):
    """P [len(recv),C] for the receivers ``recv`` (default: all, in index order); every Gaussian
    is an occluder. dirs [S,3] and Y [S,C] (SH table) are constants: P = (w V (n.w)^+) Y with V
    from ``transfer_V``."""
    d = torch.as_tensor(np.asarray(dirs, np.float64))
    Y = torch.as_tensor(np.asarray(Y, np.float64))
    n = means.shape[0]
    recv = torch.arange(n) if recv is None else torch.as_tensor(np.asarray(recv), dtype=torch.long)
    V = transfer_V(means, scales, quats, opacity, normals, dirs, recv)
    c = normals[recv] @ d.T
    w = 4.0 * math.pi / d.shape[0]
    return torch.where((c > 0).detach(), w * V * c, torch.zeros_like(c)) @ Y


def transfer_V(means, scales, quats, opacity, normals, dirs, recv=None):
    """Visibility V [len(recv),S] of the receivers' rays (0 on the rays with n.w <= 0, which are
    not traced); every Gaussian is an occluder.

    A Gaussian that no traced ray (n.w > 0) of receiver i hits contributes a factor 1 to each of
    the visibility products of receiver i, and nothing to the gradient, so after the (detached)
    hit test over all Gaussians the differentiable product of receiver i runs over the ones its
    traced rays hit."""
    d = torch.as_tensor(np.asarray(dirs, np.float64))
    n = means.shape[0]
    S = d.shape[0]
    recv = torch.arange(n) if recv is None else torch.as_tensor(np.asarray(recv), dtype=torch.long)
    R = quat_to_rot(quats)
    Sinv = R @ torch.diag_embed(1.0 / (scales * scales)) @ R.transpose(1, 2)  # [N,3,3]
    with torch.no_grad():
        traced = (normals.detach()[recv] @ d.T) > 0  # [Ni,S]: rays with n.w <= 0 contribute nothing
        chunk = max(1, (1 << 23) // max(1, len(recv) * S))
        occ_mask = torch.zeros((len(recv), n), dtype=torch.bool)
        for j0 in range(0, n, chunk):
            j1 = min(n, j0 + chunk)
            h = _hit_test(means.detach(), Sinv.detach(), means.detach()[recv], d, j0, j1)
            occ_mask[:, j0:j1] = (h & traced[:, None, :]).any(dim=2)
        occ_mask[torch.arange(len(recv)), recv] = False  # the receiver itself is no occluder
    rows = []
    for r, i in enumerate(recv.tolist()):
        occ = torch.nonzero(occ_mask[r]).flatten()
        up = traced[r]
        if occ.numel() == 0:  # nothing hit: V = 1 on every traced ray
            rows.append(torch.where(up, torch.ones(S, dtype=means.dtype), torch.zeros(S, dtype=means.dtype)))
            continue
        u = means[i][None, :] - means[occ]  # [No,3] = o - mu_j
        So = Sinv[occ]
        Sd = torch.einsum("jab,sb->jsa", So, d)  # [No,S,3]
        a = torch.einsum("sa,jsa->js", d, Sd)  # [No,S]
        b = torch.einsum("ja,jsa->js", u, Sd)  # [No,S]
        cc = torch.einsum("ja,jab,jb->j", u, So, u)  # [No]
        t = -b / a
        D2 = cc[:, None] - b * b / a
        hit = ((t > 0) & (D2 <= 9.0)).detach()
        alpha = opacity[occ][:, None] * torch.exp(-0.5 * D2)
        one_m = torch.where(hit, 1.0 - alpha, torch.ones_like(alpha))
        V = torch.prod(one_m, dim=0)  # [S]
        rows.append(torch.where(up, V, torch.zeros_like(V)))
    return torch.stack(rows)


def bounce_T(P, idx, dirs, normals, albedo, n_bounces: int = 1):
    """T [N,3,C] = P + T^1 + ... + T^n (Eq. 33-35) over a fixed index matrix idx [N,S] (-1 = no
    hit), FP64 and differentiable in P, normals and albedo: T^0_i = P_i for the three channels,
    T^k_i[c] = sum_s w max(0, n_i.w_s) (rho_j[c]/pi) T^{k-1}_j[c], j = idx[i,s], w = 4 pi/S.
    The index matrix is a discrete decision and carries no gradient; the clamp of the cosine
    has the derivative of max (zero below the horizon)."""
    idx = torch.as_tensor(np.asarray(idx), dtype=torch.int64)
    N, S = idx.shape
    d = torch.as_tensor(np.asarray(dirs, dtype=np.float64))
    w = 4.0 * math.pi / S
    valid = idx >= 0
    jj = torch.where(valid, idx, torch.zeros_like(idx))
    coef = w * torch.clamp(normals @ d.T, min=0.0) * valid  # [N,S]
    rho = albedo / math.pi  # [N,3]
    prev = P[:, None, :].expand(N, 3, P.shape[1])
    total = prev
    for _ in range(n_bounces):
        G = rho[jj][:, :, :, None] * prev[jj]  # [N,S,3,C]
        prev = (coef[:, :, None, None] * G).sum(dim=1)
        total = total + prev
    return total


def brdf_kernel(n, wi, wo, roughness, metallic):
    """k(w_i, w_o) = (1-m) + pi D F G / (4 (n.w_i)(n.w_o)) for the unit normal n/|n| (the glossy
    kernel of Eq. 15, with GGX D, Schlick F (F0 = 0.04) on w_o.h and Smith-Schlick G, k = alpha/2,
    alpha = r^2), zero unless n.w_i > 0 and n.w_o > 0 (held fixed). n [3]; wi [S,1,3], wo [1,S,3]
    broadcast; differentiable in n, roughness, metallic."""
    nu = n / torch.linalg.norm(n)
    ni = (wi * nu).sum(-1)
    no = (wo * nu).sum(-1)
    h = wi + wo
    hn = torch.linalg.norm(h, dim=-1, keepdim=True)
    h = h / torch.where(hn > 0, hn, torch.ones_like(hn))
    nh = (h * nu).sum(-1)
    oh = torch.clamp((wo * h).sum(-1), 0.0, 1.0)
    a = roughness * roughness
    a2 = a * a
    D = a2 / (math.pi * (nh * nh * (a2 - 1.0) + 1.0) ** 2)
    F = 0.04 + 0.96 * (1.0 - oh) ** 5
    kk = a / 2.0
    g = lambda x: 1.0 / (x * (1.0 - kk) + kk)  # G1(x) / x
    on = ((ni > 0) & (no > 0)).detach()
    k = (1.0 - metallic) + math.pi * 0.25 * D * F * g(torch.where(on, ni, torch.ones_like(ni))) * \
        g(torch.where(on, no, torch.ones_like(no)))
    return torch.where(on, k, torch.zeros_like(k))


def glossy_M(V, normals, roughness, metallic, dirs, Y):
    """M [R,C,C] = sum_s sum_o w^2 Y(w_s) k(w_s,w_o) (n.w_s)^+ V_s Y(w_o)^T (Eq. 40 with the in/out
    double sum over the direction set), differentiable in V [R,S], normals [R,3] (raw: the cosine
    takes n, the kernel n/|n|), roughness [R], metallic [R]."""
    d = torch.as_tensor(np.asarray(dirs, np.float64))
    Y = torch.as_tensor(np.asarray(Y, np.float64))
    S = d.shape[0]
    w = 4.0 * math.pi / S
    out = []
    for r in range(V.shape[0]):
        n = normals[r]
        K = brdf_kernel(n, d[:, None, :], d[None, :, :], roughness[r], metallic[r])  # [S_in,S_out]
        c = torch.clamp(d @ n, min=0.0)
        B = w * (K @ Y)  # [S,C]
        a = w * c * V[r]
        out.append((Y * a[:, None]).T @ B)
    return torch.stack(out)

