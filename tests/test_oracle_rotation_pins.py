"""Pins of the oracle's rotation conventions (CPU only): quaternion -> R (Eq. 2) in each of the
oracle's three restatements, and the EWA projection of a rotated, anisotropic, off-axis splat
(Eq. 3).

Each check goes through a route that does not use the quaternion-to-matrix formula under test:
Rodrigues' axis-angle formula, a rotation angle read off the quaternion with atan2, the Hamilton
product of quaternions written out here, and a central-difference Jacobian of the pinhole map.
A conjugated quaternion (R^T instead of R), a swapped (w,x,y,z) order or a transposed J W fails
at least one of them; each test also shows that the wrong convention would have changed the
result it checks.
"""
import math

import numpy as np
import pytest
import torch

from oracle import render as R
from paper_2408_03538_gb300 import scenes as S


def _hamilton(a, b):
    """Hamilton product a (x) b of (w,x,y,z) quaternions (rows)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    aw, ax, ay, az = a[..., 0], a[..., 1], a[..., 2], a[..., 3]
    bw, bx, by, bz = b[..., 0], b[..., 1], b[..., 2], b[..., 3]
    return np.stack([aw * bw - ax * bx - ay * by - az * bz,
                     aw * bx + ax * bw + ay * bz - az * by,
                     aw * by - ax * bz + ay * bw + az * bx,
                     aw * bz + ax * by - ay * bx + az * bw], axis=-1)


def _rodrigues(q):
    """Rotation matrices of (w,x,y,z) quaternions through the axis-angle reading: the rotation by
    theta = 2 atan2(|v|, w) about v / |v|, R = I + sin(theta) K + (1 - cos(theta)) K^2."""
    q = np.atleast_2d(np.asarray(q, dtype=np.float64))
    out = np.zeros((q.shape[0], 3, 3))
    for i, (w, x, y, z) in enumerate(q):
        v = np.array([x, y, z])
        nv = np.linalg.norm(v)
        if nv == 0:
            out[i] = np.eye(3)
            continue
        th = 2.0 * math.atan2(nv, w)
        k = v / nv
        K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
        out[i] = np.eye(3) + math.sin(th) * K + (1 - math.cos(th)) * (K @ K)
    return out


def _integer_quats(rng, n):
    q = rng.integers(-3, 4, size=(n, 4)).astype(np.float64)
    q[np.all(q == 0, axis=1), 0] = 1.0
    return q


def _aniso_scene(n, seed, quats):
    rng = np.random.default_rng(seed)
    means = rng.uniform(-1, 1, (n, 3))
    scales = rng.uniform(0.04, 0.45, (n, 3))  # axis ratios up to ~10:1
    normals = S.unit_vectors(rng, n)
    return S._finish(means, scales, quats, rng.uniform(0.3, 0.9, n), normals, rng.uniform(0, 1, (n, 3)))


def _band_rotation(oracle_mod, Rm, order):
    rng = np.random.default_rng(0)
    x = rng.standard_normal((64, 3))
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    Y0 = oracle_mod.sh(order, x)
    Y1 = oracle_mod.sh(order, x @ Rm.T)
    D = np.zeros((Y0.shape[1], Y0.shape[1]))
    for l in range(order + 1):
        sl = slice(l * l, (l + 1) * (l + 1))
        D[sl, sl] = np.linalg.lstsq(Y0[:, sl], Y1[:, sl], rcond=None)[0].T
    return D


def _rotated(sc, Rm, qR, compose="left"):
    q = sc.quats.astype(np.float64)
    q2 = _hamilton(qR, q) if compose == "left" else _hamilton(q, qR)
    return S.Scene(**{**sc.arrays(), "means": (sc.means.astype(np.float64) @ Rm.T).astype(np.float32),
                      "normals": (sc.normals.astype(np.float64) @ Rm.T).astype(np.float32),
                      "quats": q2.astype(np.float32)})


# signed permutation matrices (active rotations) and their quaternions, unnormalised with
# integer components: 90 deg about z, 120 deg about (1,1,1) (x->y->z->x), 90 deg about x
_PERMS = [
    (np.array([[0, -1, 0], [1, 0, 0], [0, 0, 1]], float), (1.0, 0.0, 0.0, 1.0)),
    (np.array([[0, 0, 1], [1, 0, 0], [0, 1, 0]], float), (1.0, 1.0, 1.0, 1.0)),
    (np.array([[1, 0, 0], [0, 0, -1], [0, 1, 0]], float), (1.0, 1.0, 0.0, 0.0)),
]


def test_permutation_quaternions_are_the_matrices():
    # the test's own fixtures, through Rodrigues (no quaternion-to-matrix formula involved)
    for Rm, qR in _PERMS:
        np.testing.assert_allclose(_rodrigues(np.asarray(qR) / np.linalg.norm(qR))[0], Rm, atol=1e-15)


@pytest.mark.parametrize("k", [0, 1, 2])
def test_rotation_invariance_with_rotated_anisotropic_quaternions(oracle_mod, k):
    """Rotating means, normals and directions by R and every quaternion by q_R (x) q maps P to
    D(R) P band-wise. Integer quaternions and signed permutations keep every FP32 input exact,
    so this holds to FP64 rounding; composing on the wrong side does not."""
    Rm, qR = _PERMS[k]
    rng = np.random.default_rng(40 + k)
    sc = _aniso_scene(80, 50 + k, _integer_quats(rng, 80))
    dirs = S.direction_set(128, 9)
    recv = np.arange(80)
    r1 = oracle_mod.transfer(sc, dirs, 3, recv)
    rot = _rotated(sc, Rm, qR)
    dirs2 = (dirs.astype(np.float64) @ Rm.T).astype(np.float32)
    r2 = oracle_mod.transfer(rot, dirs2, 3, recv)
    D = _band_rotation(oracle_mod, Rm, 3)
    np.testing.assert_allclose(r2["P"], r1["P"] @ D.T, atol=1e-12)
    assert np.mean(r1["hits"]) > 2  # real, anisotropic occlusion
    wrong = oracle_mod.transfer(_rotated(sc, Rm, qR, compose="right"), dirs2, 3, recv)
    assert np.max(np.abs(wrong["P"] - r1["P"] @ D.T)) > 1e-3


def test_rotation_invariance_general_rotation_with_quaternions(oracle_mod):
    rng = np.random.default_rng(61)
    qR = S.random_quats(rng, 1)[0]
    Rm = _rodrigues(qR)[0]
    sc = _aniso_scene(100, 62, S.random_quats(rng, 100))
    dirs = S.direction_set(256, 10)
    recv = np.arange(100)
    r1 = oracle_mod.transfer(sc, dirs, 3, recv)
    r2 = oracle_mod.transfer(_rotated(sc, Rm, qR), (dirs.astype(np.float64) @ Rm.T).astype(np.float32), 3, recv)
    D = _band_rotation(oracle_mod, Rm, 3)
    err = np.linalg.norm(r2["P"] - r1["P"] @ D.T, axis=1)
    clean = (r1["flags"] & 2).sum(1) + (r2["flags"] & 2).sum(1) == 0
    # inputs re-rounded to FP32 after the rotation: relative perturbations ~1e-7
    assert clean.sum() > 60
    assert np.max(err[clean]) < 1e-4


def test_rotated_occluder_visibility_closed_form(oracle_mod):
    """One Gaussian with scales (0.3, 0.1, 0.05) rotated by 30 deg about z, one unit above the
    receiver. Sigma^-1 = R diag(1/s^2) R^T is written out from cos/sin of the angle read off the
    FP32 quaternion (theta = 2 atan2(z, w)); a conjugated quaternion would put the long axis on
    the other diagonal (the sign of the xy entry)."""
    q = np.array([math.cos(math.radians(15)), 0.0, 0.0, math.sin(math.radians(15))], np.float32)
    a, b, cz = (float(v) for v in np.float32([0.3, 0.1, 0.05]))
    dist, sig = 1.0, 0.7
    sc = S._finish(np.array([[0, 0, 0], [0, 0, dist]], float), np.array([[0.05] * 3, [a, b, cz]]),
                   np.stack([[1, 0, 0, 0], q]).astype(float), np.array([0.5, sig]),
                   np.array([[0, 0, 1.0], [0, 0, -1.0]]), np.full((2, 3), 0.5))
    th = 2.0 * math.atan2(float(q[3]), float(q[0]))
    c, s = math.cos(th), math.sin(th)
    sxx = c * c / (a * a) + s * s / (b * b)
    syy = s * s / (a * a) + c * c / (b * b)
    sxy = c * s * (1 / (a * a) - 1 / (b * b))
    szz = 1 / (cz * cz)

    def expected_V(sxy_):
        Si = np.array([[sxx, sxy_, 0], [sxy_, syy, 0], [0, 0, szz]])
        u = np.array([0.0, 0.0, -dist])  # o - mu
        dd = np.einsum("sa,ab,sb->s", d, Si, d)
        ud = d @ (Si @ u)
        tstar = -ud / dd
        D2 = u @ Si @ u - ud * ud / dd
        hit = (d[:, 2] > 0) & (tstar > 0) & (D2 <= 9)
        return np.where(hit, 1 - float(sc.opacity[1]) * np.exp(-0.5 * D2), 1.0), hit

    dirs = S.direction_set(8192, 11)
    d = dirs.astype(np.float64)
    up = d[:, 2] > 0
    tr = oracle_mod.trace(sc, dirs, 2, [0])
    Vref, hit = expected_V(sxy)
    np.testing.assert_allclose(tr["V"][0][up], Vref[up], rtol=0, atol=1e-13)
    assert hit.sum() > 50
    Vconj, _ = expected_V(-sxy)
    assert np.max(np.abs(Vconj[up] - Vref[up])) > 0.05


def test_python_quaternion_formulas_match_rodrigues():
    """The numpy (oracle/__init__.py) and torch (oracle/render.py) quaternion-to-matrix formulas
    against the axis-angle route, for random unnormalised quaternions."""
    import oracle

    rng = np.random.default_rng(70)
    q = rng.standard_normal((200, 4)) * rng.uniform(0.2, 3.0, (200, 1))
    ref = _rodrigues(q / np.linalg.norm(q, axis=1, keepdims=True))
    np.testing.assert_allclose(oracle.quat_rot(q), ref, atol=1e-14)
    np.testing.assert_allclose(R.quat_to_rot(torch.as_tensor(q)).numpy(), ref, atol=1e-14)
    # and the (w,x,y,z) order: a pure 90-degree turn about z moves x to y
    np.testing.assert_allclose(oracle.quat_rot([[1.0, 0, 0, 1.0]])[0] @ [1, 0, 0], [0, 1, 0], atol=1e-15)


def test_ewa_conic_of_rotated_anisotropic_offaxis_splat():
    """Sigma' = J W Sigma W^T J^T (Eq. 3) for a rotated, anisotropic splat away from the optical
    axis under a rotated camera, against Sigma' built from a central-difference Jacobian of the
    world-to-pixel map and Sigma = R S^2 R^T with R from Rodrigues; then the 0.3 px^2 dilation
    and the inverse. The mean projects to the pinhole image of the centre."""
    cam = S.look_at_camera((1.3, -3.1, 1.7), (0.2, 0.1, 0.3), 50, 320, 240)
    rng = np.random.default_rng(71)
    means = np.array([[0.9, 0.4, 0.8], [-0.4, 0.5, 0.9], [0.6, -0.3, -0.1]])
    scales = np.array([[0.3, 0.1, 0.05], [0.05, 0.2, 0.12], [0.15, 0.02, 0.25]])
    quats = S.random_quats(rng, 3)
    pre = R.preprocess(torch.as_tensor(means), torch.as_tensor(scales), torch.as_tensor(quats), cam)
    Rw = np.asarray(cam.rot, dtype=np.float64)
    tw = np.asarray(cam.trans, dtype=np.float64)

    def pix(x):
        p = Rw @ x + tw
        return np.array([cam.fx * p[0] / p[2] + cam.cx, cam.fy * p[1] / p[2] + cam.cy])

    Rg = _rodrigues(quats)
    h = 1e-5
    for i in range(3):
        p = Rw @ means[i] + tw
        limx, limy = 1.3 * 0.5 * cam.width / cam.fx, 1.3 * 0.5 * cam.height / cam.fy
        assert abs(p[0] / p[2]) < limx and abs(p[1] / p[2]) < limy  # no clamping of J
        assert abs(p[0] / p[2]) > 0.05 and abs(p[1] / p[2]) > 0.02  # off-axis
        J = np.stack([(pix(means[i] + h * e) - pix(means[i] - h * e)) / (2 * h) for e in np.eye(3)], axis=1)
        Sig = Rg[i] @ np.diag(scales[i] ** 2) @ Rg[i].T
        cov = J @ Sig @ J.T + R.DILATION * np.eye(2)
        conic = np.linalg.inv(cov)
        got = pre["conic"][i].numpy()
        np.testing.assert_allclose(got, [conic[0, 0], conic[0, 1], conic[1, 1]], rtol=1e-7)
        np.testing.assert_allclose(pre["mean2d"][i].numpy(), pix(means[i]), rtol=1e-12)
        # a transposed camera rotation (W^T) would give a different footprint
        Jw = np.stack([(pix_t(means[i] + h * e, cam) - pix_t(means[i] - h * e, cam)) / (2 * h)
                       for e in np.eye(3)], axis=1)
        wrong = np.linalg.inv(Jw @ Sig @ Jw.T + R.DILATION * np.eye(2))
        assert np.max(np.abs(wrong - conic)) > 1e-2 * np.max(np.abs(conic))


def pix_t(x, cam):
    """The pinhole map with the camera rotation transposed (a plausible mistake)."""
    Rw = np.asarray(cam.rot, dtype=np.float64)
    p = Rw.T @ x + np.asarray(cam.trans, dtype=np.float64)
    return np.array([cam.fx * p[0] / p[2] + cam.cx, cam.fy * p[1] / p[2] + cam.cy])
