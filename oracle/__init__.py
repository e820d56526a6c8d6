"""PRTGS FP64 oracle -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously-correct CPU restatement of the PRTGS radiance-transfer precompute
and relighting (arxiv 2408.03538). Only the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. The CUDA library never imports
it, and it never imports the CUDA library: the two share no code.

Contents and the passages they follow:

* ``sh``                 real orthonormal SH by the Legendre recurrence (Eq. 8-10, Eq. 13).
* ``trace``/``transfer`` brute-force shadowed transfer vectors (Eq. 29 projected by Eq. 9),
                         the Gaussian ray-tracing weight and index matrix (Eq. 26, Sec. 4.4),
                         and the one-bounce self-transfer (Eq. 30-33).
* ``glossy``             the 16x16 glossy transfer matrix (Eq. 36-41) with the Disney-style
                         BRDF split of Eq. 15.
* ``relight``            L . T per Gaussian (Eq. 14), or L . M . Y(v) for glossy splats (Eq. 41).
* ``training_transfer``  the training-stage transfer vector for one known view (Eq. 28), and its
                         roughness / metallic derivatives by complex step.
* ``morton_lbvh``        Morton codes and the binary radix tree used as the BVH (Sec. 4.4).
* ``render`` (module)    3DGS projection (Eq. 3) and front-to-back compositing (Eq. 4), in
                         FP64 PyTorch so that autograd gives the oracle's gradients; the
                         pseudo-normal of a depth map and the normal loss (Eq. 23-25).

Every float input is promoted exactly to FP64. Readings of under-specified or garbled
passages are stated where they are used.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle_prtgs.so")
_SRC = os.path.join(_HERE, "prtgs_oracle.c")
_lib = None

RF_TRACED, RF_AMBIG_HIT, RF_AMBIG_ARGMAX = 1, 2, 4
DEFAULT_T_MIN = 2.0 ** -30


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, FP64, -ffp-contract=off, OpenMP when available)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC", _SRC, "-o",
            _LIB_PATH + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        lib.oracle_sh.argtypes = [ctypes.c_int, ctypes.c_int64, P, P]
        lib.oracle_trace.argtypes = [ctypes.c_int64, P, P, P, P, P, ctypes.c_int, P, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_int64, P, P, P, P, P, P, P, P, P]
        lib.oracle_morton_lbvh.argtypes = [ctypes.c_int64, P, ctypes.c_int, P, P, P, P, P, P]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def sh_count(order: int) -> int:
    return (order + 1) ** 2


# ------------------------------------------------------------------------------------------
# Spherical harmonics (Eq. 8-10)
# ------------------------------------------------------------------------------------------
def sh(order: int, dirs) -> np.ndarray:
    """Real orthonormal SH (Condon-Shortley phase, index l*l+l+m) of directions [n,3] -> [n,C]."""
    d = np.ascontiguousarray(np.asarray(dirs, dtype=np.float64).reshape(-1, 3))
    out = np.zeros((d.shape[0], sh_count(order)))
    rc = _load().oracle_sh(order, d.shape[0], _ptr(d), _ptr(out))
    if rc != 0:
        raise ValueError(f"oracle_sh: order {order} unsupported")
    return out


# ------------------------------------------------------------------------------------------
# Transfer (Sec. 4.4-4.5)
# ------------------------------------------------------------------------------------------
def trace(scene, dirs, order: int, recv, shadow: bool = True, bounce: bool = False, filter_t: float = 1.0,
          t_min: float = DEFAULT_T_MIN):
    """Brute-force tracing for receivers ``recv``; see prtgs_oracle.c for the outputs.

    Index-matrix candidates must have prefix transmittance >= t_min (the visibility cut-off);
    t_min = 0 gives the unrestricted argmax of Sec. 4.4."""
    lib = _load()
    recv = np.ascontiguousarray(np.asarray(recv, dtype=np.int64).reshape(-1))
    dirs = _f32(dirs)
    S = dirs.shape[0]
    C = sh_count(order)
    R = recv.size
    m, s, q, o, nrm = (_f32(scene.means), _f32(scene.scales), _f32(scene.quats), _f32(scene.opacity),
                       _f32(scene.normals))
    out = dict(P=np.zeros((R, C)), V=np.zeros((R, S)), idx=np.full((R, S), -1, np.int32),
               cand=np.full((R, S, 4), -1, np.int32), flags=np.zeros((R, S), np.int32), dV=np.zeros((R, S)),
               hits=np.zeros(R), hits_live=np.zeros(R))
    rc = lib.oracle_trace(m.shape[0], _ptr(m), _ptr(s), _ptr(q), _ptr(o), _ptr(nrm), S, _ptr(dirs), order,
                          (1 if shadow else 0) | (2 if bounce else 0), float(filter_t), float(t_min), R, _ptr(recv),
                          _ptr(out["P"]), _ptr(out["V"]), _ptr(out["idx"]), _ptr(out["cand"]), _ptr(out["flags"]),
                          _ptr(out["dV"]), _ptr(out["hits"]), _ptr(out["hits_live"]))
    if rc != 0:
        raise RuntimeError(f"oracle_trace failed: {rc}")
    return out


def _cos_weights(scene, dirs, recv):
    n = np.asarray(scene.normals, dtype=np.float64)[np.asarray(recv)]
    c = n @ np.asarray(dirs, dtype=np.float64).T
    return np.where(c > 0, c, 0.0)


def transfer(scene, dirs, order: int, recv, shadow: bool = True, bounce: bool = False, filter_t: float = 1.0,
             t_min: float = DEFAULT_T_MIN, tol: float = 1e-4, bounce_T: bool = True):
    """Transfer vectors for receivers ``recv``.

    Returns P [R,C] (Eq. 29: raw sum_s w V (n.w)^+ Y(w_s), w = 4 pi/S; albedo and 1/pi are
    applied at relight) and, with ``bounce``, T [R,3,C] = P + sum_s w (n.w_s)^+ (rho_j/pi) P_j
    with j the index-matrix entry of ray s (Eq. 33; the hit splat's own diffuse transfer
    carries its rho_j/pi, so T becomes RGB). ``allow_P``/``allow_T`` bound the change that
    flipping any flagged discrete decision (or stopping a ray at transmittance t_min) can
    cause, for use as a per-receiver tolerance widening. ``bounce_T=False`` returns the index
    matrix of a bounce trace without T (which needs P of every splat the index matrix points to).
    """
    recv = np.asarray(recv, dtype=np.int64).reshape(-1)
    S = np.asarray(dirs).shape[0]
    w = 4.0 * math.pi / S
    tr = trace(scene, dirs, order, recv, shadow, bounce, filter_t, t_min)
    Ys = sh(order, dirs)
    ynorm = np.linalg.norm(Ys, axis=1)
    c = _cos_weights(scene, dirs, recv)
    traced = (tr["flags"] & RF_TRACED) != 0
    allow_P = (w * c * ynorm[None, :] * (tr["dV"] + np.where(traced, t_min, 0.0))).sum(axis=1)
    res = dict(P=tr["P"], allow_P=allow_P, V=tr["V"], dV=tr["dV"], idx=tr["idx"], flags=tr["flags"],
               hits=tr["hits"], hits_live=tr["hits_live"], traced=traced.sum(axis=1))
    if not bounce:
        return res
    if not bounce_T:
        res.update(cand=tr["cand"])
        return res
    # receivers whose P is needed: every index-matrix entry, plus the alternatives of flagged rays
    amb = (tr["flags"] & RF_AMBIG_ARGMAX) != 0
    need = set(int(v) for v in tr["idx"][tr["idx"] >= 0].ravel())
    need.update(int(v) for v in tr["cand"][amb].ravel() if v >= 0)
    need = np.array(sorted(need), dtype=np.int64)
    Pj = {}
    if need.size:
        sub = transfer(scene, dirs, order, need, shadow=shadow, bounce=False, t_min=t_min)
        for k, j in enumerate(need):
            Pj[int(j)] = (sub["P"][k], sub["allow_P"][k])
    rho = np.asarray(scene.albedo, dtype=np.float64)
    R = recv.size
    C = sh_count(order)
    T = np.repeat(tr["P"][:, None, :], 3, axis=1).copy()
    allow_T = np.repeat(allow_P[:, None], 3, axis=1).copy()
    for r in range(R):
        for s in range(S):
            j = int(tr["idx"][r, s])
            if j >= 0:
                pj, aj = Pj[j]
                coef = w * c[r, s] * rho[j] / math.pi  # [3]
                T[r] += coef[:, None] * pj[None, :]
                allow_T[r] += coef * (aj + tol * np.linalg.norm(pj))
            if amb[r, s]:
                best = (rho[j][:, None] / math.pi) * Pj[j][0][None, :] if j >= 0 else np.zeros((3, C))
                worst = np.linalg.norm(best, axis=1)  # the "no hit" alternative
                for cj in tr["cand"][r, s]:
                    if cj < 0:
                        continue
                    alt = (rho[cj][:, None] / math.pi) * Pj[int(cj)][0][None, :]
                    worst = np.maximum(worst, np.linalg.norm(alt - best, axis=1))
                allow_T[r] += w * c[r, s] * worst
    res.update(T=T, allow_T=allow_T, cand=tr["cand"])
    return res


def unoccluded_norm(order: int) -> float:
    """||T|| of an unoccluded splat: sqrt(sum_l A_l^2 (2l+1)/(4 pi)), A = clamped-cosine constants."""
    return math.sqrt(sum(clamped_cosine_A(l) ** 2 * (2 * l + 1) / (4 * math.pi) for l in range(order + 1)))


def clamped_cosine_A(l: int) -> float:
    """SH coefficients of max(cos, 0) (Ramamoorthi & Hanrahan 2001): A_0=pi, A_1=2pi/3, A_2=pi/4,
    odd l>1 zero, even l: 2pi (-1)^(l/2-1)/((l+2)(l-1)) * l!/(2^l ((l/2)!)^2)."""
    if l == 0:
        return math.pi
    if l == 1:
        return 2 * math.pi / 3
    if l % 2 == 1:
        return 0.0
    return (2 * math.pi * (-1) ** (l // 2 - 1) / ((l + 2) * (l - 1))
            * math.factorial(l) / (2 ** l * math.factorial(l // 2) ** 2))


# ------------------------------------------------------------------------------------------
# Glossy transfer matrices (Eq. 36-41)
# ------------------------------------------------------------------------------------------
F0_DIELECTRIC = 0.04


def ggx_D(nh, alpha):
    """GGX / Trowbridge-Reitz normal distribution with alpha = roughness^2."""
    a2 = alpha * alpha
    return a2 / (math.pi * (nh * nh * (a2 - 1.0) + 1.0) ** 2)


def schlick_F(cos_oh, f0=0.04):
    """Schlick's Fresnel approximation."""
    return f0 + (1.0 - f0) * (1.0 - cos_oh) ** 5


def smith_G1(x, alpha):
    """Smith-Schlick masking for one direction, k = alpha / 2."""
    k = alpha / 2.0
    return x / (x * (1.0 - k) + k)


def brdf_kernel(n, wi, wo, roughness, metallic):
    """k(w_i, w_o) = (1-m) + pi f_s, f_s = D F G / (4 (n.w_i)(n.w_o)) (Eq. 15 times pi).

    Reading: Eq. 15 names D, F, G but not their forms. D = GGX with alpha = r^2,
    F = Schlick with F0 = 0.04 on (w_o . h), G = Smith-Schlick with k = alpha/2 for both
    directions (Burley 2012; Karis 2013). Zero unless n.w_i > 0 and n.w_o > 0. n is taken as
    n / |n|. Arrays broadcast: wi [..., 3], wo [..., 3].
    """
    a = roughness * roughness
    # the BRDF takes the unit normal: an FP32 normal is unit only to rounding, and near a sharp
    # GGX peak 1 - (n.h)^2 would turn that 1e-7 into a relative change of 1e-4 in D
    n = n / np.linalg.norm(n, axis=-1, keepdims=True)
    ni = (wi * n).sum(-1)
    no = (wo * n).sum(-1)
    h = wi + wo
    hn = np.linalg.norm(h, axis=-1, keepdims=True)
    h = h / np.where(hn > 0, hn, 1.0)
    nh = (h * n).sum(-1)
    oh = np.clip((wo * h).sum(-1), 0.0, 1.0)
    with np.errstate(divide="ignore", invalid="ignore"):
        fs = ggx_D(nh, a) * schlick_F(oh, F0_DIELECTRIC) * smith_G1(ni, a) * smith_G1(no, a) / (4.0 * ni * no)
    k = (1.0 - metallic) + math.pi * fs
    return np.where((no > 0) & (ni > 0), k, 0.0)


def glossy(scene, dirs, order: int, recv, V, allow_V=None):
    """M[a,b] = sum_s sum_o w^2 Y_a(w_s) k(w_s,w_o) (n.w_s)^+ V_s Y_b(w_o) (Eq. 40 with the
    in/out double sum over the same direction set, P = S outgoing samples)."""
    recv = np.asarray(recv, dtype=np.int64).reshape(-1)
    d = np.asarray(dirs, dtype=np.float64)
    S = d.shape[0]
    w = 4.0 * math.pi / S
    Y = sh(order, d)
    C = Y.shape[1]
    M = np.zeros((recv.size, C, C))
    allow = np.zeros(recv.size)
    for r, i in enumerate(recv):
        n = np.asarray(scene.normals[i], dtype=np.float64)
        K = brdf_kernel(n[None, None, :], d[:, None, :], d[None, :, :], float(scene.roughness[i]),
                        float(scene.metallic[i]))  # [S_in, S_out]
        c = np.maximum(d @ n, 0.0)
        B = w * (K @ Y)  # [S_in, C]: sum_o w k(s,o) Y_b(o)
        a = w * c * V[r]
        M[r] = (Y * a[:, None]).T @ B
        if allow_V is not None:
            allow[r] = np.sum(w * c * allow_V[r] * np.linalg.norm(Y, axis=1) * np.linalg.norm(B, axis=1))
    return M, allow


# ------------------------------------------------------------------------------------------
# Training-stage transfer for one known view direction (Sec. 4.5, Eq. 28)
# ------------------------------------------------------------------------------------------
def view_dirs(means, cam_pos):
    """v_i = (cam_pos - mu_i) / |cam_pos - mu_i|: the direction from a splat to the camera."""
    v = np.asarray(cam_pos, dtype=np.float64)[None, :] - np.asarray(means, dtype=np.float64)
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def training_transfer(scene, dirs, order: int, recv, V, cam_pos, specular: bool = True, roughness=None,
                      metallic=None):
    """t_i[c] = sum_s w k_i(w_s, v_i) (n_i.w_s)^+ V_is Y_c(w_s), w = 4 pi / S (Eq. 28).

    Reading: Eq. 28 is printed as (f_s(w_i,v) + f_d)(v.n)V(v,x), but the text defines the
    transfer on the sphere of incident directions w_i, so the cosine and the visibility are
    read as those of w_i; the view direction v enters through the BRDF only. The BRDF is the
    same k = (1-m) + pi f_s as the glossy matrices (Eq. 15 times pi; albedo and 1/pi applied
    at relight, as for P), so with f_s = 0 (``specular=False``) and m = 0 the vector is
    exactly the diffuse transfer P of Eq. 29. v_i = normalize(cam_pos - mu_i). No bounce term
    (the paper trades the indirect light's accuracy for speed during training).
    V [R,S] is the visibility of the receivers ``recv`` (as ``trace`` returns it).
    ``roughness`` / ``metallic`` [R] override the scene's (complex values are allowed: they
    flow through k, which is what ``training_transfer_grad`` uses).
    """
    recv = np.asarray(recv, dtype=np.int64).reshape(-1)
    d = np.asarray(dirs, dtype=np.float64)
    S = d.shape[0]
    w = 4.0 * math.pi / S
    Y = sh(order, d)
    v = view_dirs(np.asarray(scene.means, dtype=np.float64)[recv], cam_pos)
    rough = np.asarray(scene.roughness, dtype=np.float64)[recv] if roughness is None else roughness
    metal = np.asarray(scene.metallic, dtype=np.float64)[recv] if metallic is None else metallic
    dtype = np.result_type(np.asarray(rough), np.asarray(metal), np.float64)
    t = np.zeros((recv.size, Y.shape[1]), dtype=dtype)
    for r, i in enumerate(recv):
        n = np.asarray(scene.normals[i], dtype=np.float64)
        c = np.maximum(d @ n, 0.0)
        if specular:
            k = brdf_kernel(n[None, :], d, v[r][None, :], rough[r], metal[r])  # [S]
        else:
            nu = n / np.linalg.norm(n)
            k = np.where((d @ nu > 0) & (float(v[r] @ nu) > 0), 1.0 - metal[r], 0.0)
        t[r] = (w * k * c * np.asarray(V[r], dtype=np.float64)) @ Y
    return t


def training_transfer_grad(scene, dirs, order: int, recv, V, cam_pos, dT, h: float = 1e-30):
    """d(sum_c dT[r,c] t_r[c]) / d roughness_r and / d metallic_r for each receiver r of
    ``training_transfer``: complex-step differentiation (Squire and Trapp 1998), exact to
    rounding since k is analytic in both; t_r depends only on receiver r's own parameters, so
    one complex evaluation gives every receiver's derivative."""
    recv = np.asarray(recv, dtype=np.int64).reshape(-1)
    dT = np.asarray(dT, dtype=np.float64)
    rough = np.asarray(scene.roughness, dtype=np.float64)[recv]
    metal = np.asarray(scene.metallic, dtype=np.float64)[recv]
    tr = training_transfer(scene, dirs, order, recv, V, cam_pos, roughness=rough + 1j * h, metallic=metal)
    tm = training_transfer(scene, dirs, order, recv, V, cam_pos, roughness=rough, metallic=metal + 1j * h)
    return (dT * tr.imag).sum(1) / h, (dT * tm.imag).sum(1) / h


def multi_bounce(scene, dirs, order: int, tr, n_bounces: int, tol: float = 1e-4):
    """n-bounce self-transfer (Eq. 34-35) over an index matrix.

    ``tr`` is ``transfer(scene, dirs, order, np.arange(N), bounce=True)`` (every Gaussian a
    receiver, so every index target is present) or any dict with the same P, allow_P, idx,
    flags, cand. With T^0 = P (the diffuse transfer, the same for the three channels):
        T^k_i = sum_s w (n_i.w_s)^+ (rho_j / pi) T^{k-1}_j,   j = idx[i, s] >= 0, per channel,
    and the total is T = P + sum_{k=1..n} T^k [N,3,C] (Eq. 35). One bounce gives Eq. 33.
    The allowance [N,3] carries each bounce's: the previous bounce's allowance and relative
    tolerance through the weights, plus, for a ray whose argmax is flagged, the largest change
    switching to another candidate (or to no hit) would make.
    """
    P = np.asarray(tr["P"], dtype=np.float64)
    idx = np.asarray(tr["idx"])
    N, S = idx.shape
    w = 4.0 * math.pi / S
    c = _cos_weights(scene, dirs, np.arange(N))
    rho = np.asarray(scene.albedo, dtype=np.float64) / math.pi  # [N,3]
    valid = idx >= 0
    jj = np.where(valid, idx, 0)
    coef = w * c * valid  # [N,S]
    amb = np.nonzero((np.asarray(tr["flags"]) & RF_AMBIG_ARGMAX) != 0)
    cand = np.asarray(tr["cand"]) if "cand" in tr else None
    prev = np.repeat(P[:, None, :], 3, axis=1)
    aprev = np.repeat(np.asarray(tr["allow_P"], dtype=np.float64)[:, None], 3, axis=1)
    total, atot = prev.copy(), aprev.copy()
    for _ in range(n_bounces):
        G = rho[jj][:, :, :, None] * prev[jj]  # [N,S,3,C]: (rho_j/pi) T^{k-1}_j
        cur = (coef[:, :, None, None] * G).sum(axis=1)
        nrm = np.linalg.norm(prev, axis=2)  # [N,3]
        acur = (coef[:, :, None] * rho[jj] * (aprev[jj] + tol * nrm[jj])).sum(axis=1)
        for i, sidx in zip(*amb):
            best = G[i, sidx] if valid[i, sidx] else np.zeros_like(G[i, sidx])
            worst = np.linalg.norm(best, axis=1)
            for cj in (cand[i, sidx] if cand is not None else ()):
                if cj >= 0:
                    worst = np.maximum(worst, np.linalg.norm(rho[cj][:, None] * prev[cj] - best, axis=1))
            acur[i] += w * c[i, sidx] * worst
        total += cur
        atot += acur
        prev, aprev = cur, acur
    return total, atot


# ------------------------------------------------------------------------------------------
# Relight (Eq. 14, Eq. 41)
# ------------------------------------------------------------------------------------------
def relight(T, albedo, L, glossy_ids=None, M=None, means=None, cam_pos=None, order=None):
    """colors[k,N,3] = (rho/pi) * (T . L_k) per channel (Eq. 14 with f_d = rho/pi).

    T is [N,C] (same transfer for all channels) or [N,3,C]. Glossy splats (``glossy_ids``)
    use t_eff[a] = sum_b M[a,b] Y_b(v), v = normalize(cam_pos - mu) (Eq. 41).
    """
    T = np.asarray(T, dtype=np.float64)
    L = np.asarray(L, dtype=np.float64)
    rho = np.asarray(albedo, dtype=np.float64)
    if T.ndim == 2:
        T = np.repeat(T[:, None, :], 3, axis=1)
    else:
        T = T.copy()
    if glossy_ids is not None and len(glossy_ids):
        mu = np.asarray(means, dtype=np.float64)[glossy_ids]
        v = np.asarray(cam_pos, dtype=np.float64)[None, :] - mu
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        Yv = sh(order if order is not None else int(round(math.sqrt(T.shape[2]))) - 1, v)
        teff = np.einsum("gab,gb->ga", np.asarray(M, dtype=np.float64), Yv)
        T[glossy_ids] = teff[:, None, :]
    dot = np.einsum("nch,kch->knc", T, L)
    return dot * (rho / math.pi)[None]


# ------------------------------------------------------------------------------------------
# Morton codes + radix tree (Sec. 4.4 BVH)
# ------------------------------------------------------------------------------------------
def morton_lbvh(means, offsets=None):
    means = _f32(means)
    n = means.shape[0]
    if offsets is None:
        offsets = np.array([0, n], dtype=np.int64)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    B = offsets.size - 1
    codes = np.zeros(n, np.uint32)
    keys = np.zeros(n, np.uint64)
    order = np.zeros(n, np.int32)
    children = np.zeros((max(n - 1, 1), 2), np.int32)
    roots = np.zeros(B, np.int32)
    rc = _load().oracle_morton_lbvh(n, _ptr(means), B, _ptr(offsets), _ptr(codes), _ptr(keys), _ptr(order),
                                    _ptr(children), _ptr(roots))
    if rc != 0:
        raise RuntimeError("oracle_morton_lbvh failed")
    return dict(codes=codes, keys=keys, order=order, children=children[: max(n - 1, 0)], roots=roots)


def aabb_3sigma(scene):
    """Exact FP64 3-sigma AABBs [N,6] (lo xyz, hi xyz): half-extent_a = 3 sqrt(Sigma_aa)."""
    R = quat_rot(scene.quats)
    s2 = np.asarray(scene.scales, dtype=np.float64) ** 2
    sig_diag = np.einsum("nak,nk->na", R * R, s2)
    h = 3.0 * np.sqrt(sig_diag)
    mu = np.asarray(scene.means, dtype=np.float64)
    return np.concatenate([mu - h, mu + h], axis=1)


def quat_rot(quats):
    """Rotation matrices [N,3,3] of (w,x,y,z) quaternions (normalised first), Eq. 2's R."""
    q = np.asarray(quats, dtype=np.float64)
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], axis=1)


def norm_err(gpu, ref, floor):
    """Per-row norm-wise error ||gpu - ref|| / max(||ref||, floor)."""
    g = np.asarray(gpu, dtype=np.float64).reshape(len(gpu), -1)
    r = np.asarray(ref, dtype=np.float64).reshape(len(ref), -1)
    return np.linalg.norm(g - r, axis=1) / np.maximum(np.linalg.norm(r, axis=1), floor)
