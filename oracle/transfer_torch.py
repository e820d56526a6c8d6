"""FP64 PyTorch restatement of the shadowed transfer P -- TEST INFRASTRUCTURE ONLY.

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


def transfer_P(means, scales, quats, opacity, normals, dirs, Y, recv=None):
    """P [len(recv),C] for the receivers ``recv`` (default: all, in index order); every Gaussian
    is an occluder. dirs [S,3] and Y [S,C] (SH table) are constants."""
    d = torch.as_tensor(np.asarray(dirs, np.float64))
    Y = torch.as_tensor(np.asarray(Y, np.float64))
    n = means.shape[0]
    S = d.shape[0]
    recv = torch.arange(n) if recv is None else torch.as_tensor(np.asarray(recv), dtype=torch.long)
    R = quat_to_rot(quats)
    Sinv = R @ torch.diag_embed(1.0 / (scales * scales)) @ R.transpose(1, 2)  # [N,3,3]
    u = means[recv][:, None, :] - means[None, :, :]  # [Ni,Nj,3] = o - mu_j
    Sd = torch.einsum("jab,sb->jsa", Sinv, d)  # [Nj,S,3]
    a = torch.einsum("sa,jsa->js", d, Sd)  # [Nj,S]
    b = torch.einsum("ija,jsa->ijs", u, Sd)  # [Ni,Nj,S]
    cc = torch.einsum("ija,jab,ijb->ij", u, Sinv, u)  # [Ni,Nj]
    t = -b / a[None]
    D2 = cc[:, :, None] - b * b / a[None]
    hit = ((t > 0) & (D2 <= 9.0)).detach()
    hit = hit & (recv[:, None] != torch.arange(n)[None, :])[:, :, None]
    alpha = opacity[None, :, None] * torch.exp(-0.5 * D2)
    one_m = torch.where(hit, 1.0 - alpha, torch.ones_like(alpha))
    V = torch.prod(one_m, dim=1)  # [Ni,S]
    c = normals[recv] @ d.T  # [Ni,S]
    up = (c > 0).detach()
    w = 4.0 * math.pi / S
    contrib = torch.where(up, w * V * c, torch.zeros_like(c))
    return contrib @ Y
