"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics (CPU only).

Each test checks the oracle against something other than itself: a closed form, an
identity, a textbook result or brute force on tiny inputs, chosen so that a dropped term,
wrong sign, wrong index or transposed operand fails at least one of them.
"""
import math

import numpy as np
import pytest

from paper_2408_03538_gb300 import scenes as S


def _sc(means, scales, opacity, normals, quats=None, albedo=None):
    n = len(means)
    quats = quats if quats is not None else np.tile([1.0, 0.0, 0.0, 0.0], (n, 1))
    albedo = albedo if albedo is not None else np.full((n, 3), 0.5)
    return S._finish(np.asarray(means, float), np.asarray(scales, float), np.asarray(quats, float),
                     np.asarray(opacity, float), np.asarray(normals, float), np.asarray(albedo, float))


# ------------------------------------------------------------------------------------------
# Spherical harmonics (Eq. 8-10, Eq. 13)
# ------------------------------------------------------------------------------------------
def _sh_cartesian(d):
    """Textbook Cartesian real SH, l <= 3 (e.g. Sloan, 'Stupid Spherical Harmonics Tricks',
    2008, Appendix A2), Condon-Shortley phase, index l*l+l+m."""
    x, y, z = d[:, 0], d[:, 1], d[:, 2]
    pi = math.pi
    return np.stack([
        np.full_like(x, 0.5 / math.sqrt(pi)),
        -math.sqrt(3 / (4 * pi)) * y, math.sqrt(3 / (4 * pi)) * z, -math.sqrt(3 / (4 * pi)) * x,
        0.5 * math.sqrt(15 / pi) * x * y, -0.5 * math.sqrt(15 / pi) * y * z,
        0.25 * math.sqrt(5 / pi) * (3 * z * z - 1), -0.5 * math.sqrt(15 / pi) * x * z,
        0.25 * math.sqrt(15 / pi) * (x * x - y * y),
        -0.25 * math.sqrt(35 / (2 * pi)) * y * (3 * x * x - y * y), 0.5 * math.sqrt(105 / pi) * x * y * z,
        -0.25 * math.sqrt(21 / (2 * pi)) * y * (5 * z * z - 1), 0.25 * math.sqrt(7 / pi) * (5 * z ** 3 - 3 * z),
        -0.25 * math.sqrt(21 / (2 * pi)) * x * (5 * z * z - 1), 0.25 * math.sqrt(105 / pi) * (x * x - y * y) * z,
        -0.25 * math.sqrt(35 / (2 * pi)) * x * (x * x - 3 * y * y)], axis=1)


def test_sh_matches_cartesian_closed_forms(oracle_mod):
    rng = np.random.default_rng(1)
    d = rng.standard_normal((2000, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    np.testing.assert_allclose(oracle_mod.sh(3, d), _sh_cartesian(d), atol=1e-13, rtol=0)
    assert abs(oracle_mod.sh(0, d[:1])[0, 0] - 1 / (2 * math.sqrt(math.pi))) < 1e-15


def test_sh_orthonormal_by_exact_quadrature(oracle_mod):
    # Gauss-Legendre in z times a uniform azimuth grid integrates products of l<=6 SH exactly
    z, wz = np.polynomial.legendre.leggauss(16)
    nphi = 32
    phi = (np.arange(nphi) + 0.5) * 2 * math.pi / nphi
    zz, pp = np.meshgrid(z, phi, indexing="ij")
    r = np.sqrt(1 - zz ** 2)
    d = np.stack([r * np.cos(pp), r * np.sin(pp), zz], -1).reshape(-1, 3)
    w = (wz[:, None] * np.full(nphi, 2 * math.pi / nphi)[None, :]).reshape(-1)
    for order in (1, 2, 3, 6):
        Y = oracle_mod.sh(order, d)
        G = (Y * w[:, None]).T @ Y
        np.testing.assert_allclose(G, np.eye(Y.shape[1]), atol=1e-12)


def test_sh_orthonormal_monte_carlo(oracle_mod):
    rng = np.random.default_rng(2)
    n = 1 << 20
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    Y = oracle_mod.sh(3, d)
    G = 4 * math.pi / n * (Y.T @ Y)
    assert np.max(np.abs(G - np.eye(16))) < 5 / math.sqrt(n) * 4 * math.pi * 0.5


# ------------------------------------------------------------------------------------------
# Direction set and unoccluded transfer (Eq. 29 with V = 1)
# ------------------------------------------------------------------------------------------
def test_direction_set_is_unit_and_equal_area():
    d = S.direction_set(4096, 5).astype(np.float64)
    assert np.all(np.abs(np.linalg.norm(d, axis=1) - 1) < 1e-6)
    # one direction per equal-area band of z (FP32 rounding may move a point onto a band edge)
    k = (1 - d[:, 2]) * 4096 / 2
    assert np.all(np.abs(np.sort(k) - (np.arange(4096) + 0.5)) <= 0.5 + 1e-3)


@pytest.mark.parametrize("order", [2, 3, 6])
def test_unoccluded_transfer_is_clamped_cosine(oracle_mod, order):
    """An unoccluded splat's transfer is A_l Y_lm(n) (Ramamoorthi & Hanrahan 2001)."""
    rng = np.random.default_rng(order)
    nrm = rng.standard_normal((3, 3))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    dirs = S.direction_set(1 << 18, 11)
    # three receivers far apart from each other: nothing occludes anything
    sc = _sc([[0, 0, 0], [100, 0, 0], [0, 100, 0]], np.full((3, 3), 0.01), [0.5] * 3, nrm)
    r = oracle_mod.transfer(sc, dirs, order, [0, 1, 2])
    A = np.array([oracle_mod.clamped_cosine_A(l) for l in range(order + 1) for _ in range(2 * l + 1)])
    ref = A[None, :] * oracle_mod.sh(order, nrm)
    assert np.max(np.abs(r["P"] - ref)) < 2e-4
    assert np.all(r["hits"] == 0)


def test_clamped_cosine_constants():
    import oracle

    assert oracle.clamped_cosine_A(0) == pytest.approx(math.pi)
    assert oracle.clamped_cosine_A(1) == pytest.approx(2 * math.pi / 3)
    assert oracle.clamped_cosine_A(2) == pytest.approx(math.pi / 4)
    assert oracle.clamped_cosine_A(3) == 0.0
    assert oracle.clamped_cosine_A(4) == pytest.approx(-math.pi / 24)
    # and numerically: 2 pi int_0^1 z P_l(z) dz Y_l0-normalisation
    for l in range(5):
        z, w = np.polynomial.legendre.leggauss(64)
        z, w = 0.5 * (z + 1), 0.5 * w
        Pl = np.polynomial.legendre.legval(z, [0] * l + [1])
        A_num = 2 * math.pi * np.sum(w * z * Pl)
        assert A_num == pytest.approx(oracle.clamped_cosine_A(l), abs=1e-12)


# ------------------------------------------------------------------------------------------
# Transmittance (Eq. 27 read as the maximum along the ray; Eq. 4 along a ray)
# ------------------------------------------------------------------------------------------
def _axis_occluder_D2(dirs, dist, a, b, c):
    """Closed form D^2 of an axis-aligned occluder with scales (a,b,c) at (0,0,dist) seen from
    the origin: the whitened cross product |u' x d'|^2 / |d'|^2."""
    dx, dy, dz = dirs[:, 0], dirs[:, 1], dirs[:, 2]
    q = dx * dx / (a * a) + dy * dy / (b * b)
    return dist * dist * q / (c * c * (q + dz * dz / (c * c)))


@pytest.mark.parametrize("scales", [(0.2, 0.2, 0.2), (0.3, 0.1, 0.05)])
def test_single_occluder_visibility_closed_form(oracle_mod, scales):
    dist, sig = 1.0, 0.7
    sc = _sc([[0, 0, 0], [0, 0, dist]], [[0.05] * 3, scales], [0.5, sig], [[0, 0, 1], [0, 0, -1]])
    dirs = S.direction_set(4096, 3)
    tr = oracle_mod.trace(sc, dirs, 2, [0])
    d = dirs.astype(np.float64)
    D2 = _axis_occluder_D2(d, dist, *sc.scales[1].astype(np.float64))
    up = d[:, 2] > 0
    hit = up & (D2 <= 9)
    Vref = np.where(hit, 1 - float(sc.opacity[1]) * np.exp(-0.5 * D2), 1.0)
    np.testing.assert_allclose(tr["V"][0][up], Vref[up], rtol=0, atol=1e-13)
    assert hit.sum() > 20
    assert np.all(tr["V"][0][~up] == 0)  # untraced


def test_single_occluder_transfer_axisymmetric_quadrature(oracle_mod):
    """m=0 coefficients against an adaptive 1-D theta quadrature of the axisymmetric integrand."""
    from scipy.integrate import quad

    dist, s, sig = 1.0, 0.25, 0.8
    sc = _sc([[0, 0, 0], [0, 0, dist]], [[0.05] * 3, [s] * 3], [0.5, sig], [[0, 0, 1], [0, 0, -1]])
    dirs = S.direction_set(1 << 18, 9)
    P = oracle_mod.transfer(sc, dirs, 3, [0])["P"][0]
    thc = math.asin(min(1.0, 3 * s / dist))

    def V(th):
        return 1 - sig * math.exp(-0.5 * (dist * math.sin(th) / s) ** 2) if th <= thc else 1.0

    for l in range(4):
        Pl = lambda th: np.polynomial.legendre.legval(math.cos(th), [0] * l + [1])
        K = math.sqrt((2 * l + 1) / (4 * math.pi))
        f = lambda th: 2 * math.pi * V(th) * math.cos(th) * K * Pl(th) * math.sin(th)
        ref = quad(f, 0, thc, epsabs=1e-13, limit=200)[0] + quad(f, thc, math.pi / 2, epsabs=1e-13, limit=200)[0]
        assert P[l * l + l] == pytest.approx(ref, abs=3e-4)
    # m != 0 vanish by symmetry (to the direction set's quadrature noise)
    assert np.max(np.abs(np.delete(P, [0, 2, 6, 12]))) < 3e-4


def test_two_occluders_multiply_and_order_does_not_matter(oracle_mod):
    occ = [[0.05, 0.02, 1.0], [-0.03, 0.04, 2.0]]
    base = dict(scales=[[0.05] * 3, [0.3] * 3, [0.4] * 3], opacity=[0.5, 0.6, 0.9],
                normals=[[0, 0, 1], [0, 0, -1], [0, 0, -1]])
    dirs = S.direction_set(2048, 4)
    both = oracle_mod.trace(_sc([[0, 0, 0]] + occ, **base), dirs, 2, [0])["V"][0]
    a = oracle_mod.trace(_sc([[0, 0, 0], occ[0], [50, 50, 50]], **base), dirs, 2, [0])["V"][0]
    b = oracle_mod.trace(_sc([[0, 0, 0], [50, 50, 50], occ[1]], **base), dirs, 2, [0])["V"][0]
    np.testing.assert_allclose(both, a * b, rtol=1e-14, atol=0)
    swapped = _sc([[0, 0, 0], occ[1], occ[0]], scales=[base["scales"][0], base["scales"][2], base["scales"][1]],
                  opacity=[0.5, 0.9, 0.6], normals=base["normals"])
    np.testing.assert_allclose(oracle_mod.trace(swapped, dirs, 2, [0])["V"][0], both, rtol=1e-14, atol=0)
    assert np.sum(both < 1) > 10


def test_occluder_behind_or_around_origin_is_ignored(oracle_mod):
    # occluder below the receiver (t* < 0 for every upward ray), and the receiver itself
    sc = _sc([[0, 0, 0], [0, 0, -0.5]], [[0.2] * 3, [0.3] * 3], [0.9, 0.9], [[0, 0, 1], [0, 0, 1]])
    dirs = S.direction_set(1024, 8)
    tr = oracle_mod.trace(sc, dirs, 2, [0])
    up = dirs[:, 2] > 0
    assert np.all(tr["V"][0][up] == 1.0)


def _signed_perms():
    return [np.array([[0, -1, 0], [1, 0, 0], [0, 0, 1]], float),  # 90 deg about z
            np.array([[0, 0, 1], [1, 0, 0], [0, 1, 0]], float),   # cyclic axes
            np.array([[1, 0, 0], [0, 0, -1], [0, 1, 0]], float)]  # 90 deg about x


def _band_rotation(oracle_mod, Rm, order):
    """SH rotation matrix D(R), fitted band by band from Y_l(R x) = D_l Y_l(x) on many points."""
    rng = np.random.default_rng(0)
    x = rng.standard_normal((64, 3))
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    Y0 = oracle_mod.sh(order, x)
    Y1 = oracle_mod.sh(order, x @ Rm.T)
    C = Y0.shape[1]
    D = np.zeros((C, C))
    for l in range(order + 1):
        sl = slice(l * l, (l + 1) * (l + 1))
        D[sl, sl] = np.linalg.lstsq(Y0[:, sl], Y1[:, sl], rcond=None)[0].T
    return D


@pytest.mark.parametrize("k", [0, 1, 2])
def test_rotation_invariance_exact(oracle_mod, k):
    """Rotating scene and direction set by R maps P to D(R) P band-wise (signed permutations
    keep every FP32 input exact, so this holds to FP64 rounding)."""
    Rm = _signed_perms()[k]
    sc = S.isotropic_scene(96, 77)
    sc.scales *= 4  # more occlusion
    dirs = S.direction_set(128, 5)
    recv = np.arange(96)
    P = oracle_mod.transfer(sc, dirs, 3, recv)["P"]
    rot = S.Scene(**{**sc.arrays(), "means": (sc.means @ Rm.T).astype(np.float32),
                     "normals": (sc.normals @ Rm.T).astype(np.float32)})
    P2 = oracle_mod.transfer(rot, (dirs @ Rm.T).astype(np.float32), 3, recv)["P"]
    D = _band_rotation(oracle_mod, Rm, 3)
    np.testing.assert_allclose(P2, P @ D.T, atol=1e-12)
    assert np.mean(oracle_mod.transfer(sc, dirs, 3, recv)["hits"]) > 0


def test_rotation_invariance_general(oracle_mod):
    rng = np.random.default_rng(3)
    Rm = S.random_rotation_matrices(rng, 1)[0]
    sc = S.isotropic_scene(128, 78)
    sc.scales *= 3
    dirs = S.direction_set(256, 6)
    recv = np.arange(128)
    r1 = oracle_mod.transfer(sc, dirs, 3, recv)
    rot = S.Scene(**{**sc.arrays(), "means": (sc.means.astype(float) @ Rm.T).astype(np.float32),
                     "normals": (sc.normals.astype(float) @ Rm.T).astype(np.float32)})
    r2 = oracle_mod.transfer(rot, (dirs.astype(float) @ Rm.T).astype(np.float32), 3, recv)
    D = _band_rotation(oracle_mod, Rm, 3)
    err = np.linalg.norm(r2["P"] - r1["P"] @ D.T, axis=1)
    clean = (r1["flags"] & 2).sum(1) + (r2["flags"] & 2).sum(1) == 0
    # inputs re-rounded to FP32 after rotation: relative perturbations ~1e-7
    assert np.max(err[clean]) < 1e-4
    assert clean.sum() > 100


# ------------------------------------------------------------------------------------------
# Index matrix and one-bounce self-transfer (Eq. 26, Sec. 4.4, Eq. 30-33)
# ------------------------------------------------------------------------------------------
def test_index_matrix_weight_closed_form(oracle_mod):
    up = np.array([[0, 0, 1.0], [0.6, 0, 0.8], [0, 0.6, 0.8]], np.float32)
    # A at height 1 (opacity sA), B at height 2 (opacity 0.9), both facing down
    for sA, expect in ((0.3, 2), (0.6, 1)):
        sc = _sc([[0, 0, 0], [0, 0, 1], [0, 0, 2]], [[0.05] * 3, [0.1] * 3, [0.1] * 3], [0.5, sA, 0.9],
                 [[0, 0, 1], [0, 0, -1], [0, 0, -1]])
        tr = oracle_mod.trace(sc, up, 2, [0], bounce=True)
        # W_A = sA, W_B = 0.9 (1 - sA) on the straight-up ray
        assert tr["idx"][0, 0] == expect
        assert tr["idx"][0, 1] == -1 and tr["idx"][0, 2] == -1  # those rays miss both
    # filter t = 0.8: A (prefix T = 1) is filtered out, B (prefix T = 0.7) is kept
    sc = _sc([[0, 0, 0], [0, 0, 1], [0, 0, 2]], [[0.05] * 3, [0.1] * 3, [0.1] * 3], [0.5, 0.3, 0.9],
             [[0, 0, 1], [0, 0, -1], [0, 0, -1]])
    assert oracle_mod.trace(sc, up, 2, [0], bounce=True, filter_t=0.8)["idx"][0, 0] == 2
    # a front-facing splat behind a near-opaque stack: it is the argmax, unless its prefix
    # transmittance is below the cut-off t_min
    stack = [[0, 0, 0.5 + 0.01 * k] for k in range(6)]
    sc = _sc([[0, 0, 0]] + stack + [[0, 0, 2]], [[0.05] * 3] + [[0.1] * 3] * 6 + [[0.1] * 3],
             [0.5] + [0.9] * 6 + [0.9], [[0, 0, 1]] + [[0, 0, 1]] * 6 + [[0, 0, -1]])
    # prefix in front of the last splat: 0.1^6 = 1e-6
    assert oracle_mod.trace(sc, up, 2, [0], bounce=True, t_min=0.0)["idx"][0, 0] == 7
    assert oracle_mod.trace(sc, up, 2, [0], bounce=True, t_min=1e-7)["idx"][0, 0] == 7
    assert oracle_mod.trace(sc, up, 2, [0], bounce=True, t_min=1e-5)["idx"][0, 0] == -1
    # back-facing hits have zero weight: no index
    sc = _sc([[0, 0, 0], [0, 0, 1]], [[0.05] * 3, [0.1] * 3], [0.5, 0.9], [[0, 0, 1], [0, 0, 1]])
    assert oracle_mod.trace(sc, up, 2, [0], bounce=True)["idx"][0, 0] == -1


def test_index_matrix_flags_a_reorder_past_the_winner(oracle_mod):
    """Hits A (front-facing, opacity 0.3, the winner: W = 0.3), B and X (back-facing) and Y
    (front-facing, opacity 0.9) up the z axis. In order, W_Y = 0.9 (0.7)(0.8)(0.5) = 0.252 < W_A;
    placed in front of X it would be 0.9 (0.7)(0.8) = 0.504 > W_A. With Y a rounding step behind
    X the argmax is open (flagged); with Y well behind X it is not."""
    up = np.array([[0, 0, 1.0]], np.float32)
    for zy, flagged in ((2.0 + 1e-6, True), (2.5, False)):
        sc = _sc([[0, 0, 0], [0, 0, 1], [0, 0, 1.5], [0, 0, 2], [0, 0, zy]], [[0.05] * 3] + [[0.1] * 3] * 4,
                 [0.5, 0.3, 0.2, 0.5, 0.9], [[0, 0, 1], [0, 0, -1], [0, 0, 1], [0, 0, 1], [0, 0, -1]])
        tr = oracle_mod.trace(sc, up, 1, [0], bounce=True)
        assert tr["idx"][0, 0] == 1
        assert bool(tr["flags"][0, 0] & oracle_mod.RF_AMBIG_ARGMAX) == flagged
        assert not tr["flags"][0, 0] & oracle_mod.RF_AMBIG_HIT


def test_bounce_against_closed_form_disc(oracle_mod):
    """Wide facing disc above the receiver: every ray within its 3-sigma footprint records it."""
    a, b, c, h, sig = 1.0, 0.8, 0.05, 1.0, 0.5
    rho = np.array([0.5, 0.2, 0.8])
    sc = _sc([[0, 0, 0], [0, 0, h]], [[0.05] * 3, [a, b, c]], [0.5, sig], [[0, 0, 1], [0, 0, -1]],
             albedo=[[0.3, 0.3, 0.3], rho])
    dirs = S.direction_set(512, 12)
    r = oracle_mod.transfer(sc, dirs, 3, [0], bounce=True)
    d = dirs.astype(np.float64)
    D2 = _axis_occluder_D2(d, h, *sc.scales[1].astype(np.float64))
    hit = (d[:, 2] > 0) & (D2 <= 9)
    np.testing.assert_array_equal(r["idx"][0], np.where(hit, 1, -1))
    P1 = oracle_mod.transfer(sc, dirs, 3, [1])["P"][0]
    w = 4 * math.pi / 512
    bounce = (w * d[hit, 2]).sum() * (sc.albedo[1].astype(np.float64)[:, None] / math.pi) * P1[None, :]
    np.testing.assert_allclose(r["T"][0] - r["P"][0][None, :], bounce, atol=1e-14)


def test_bounce_linear_in_albedo_and_zero_without_it(oracle_mod):
    sc = S.isotropic_scene(200, 31)
    sc.scales *= 3
    dirs = S.direction_set(64, 2)
    recv = np.arange(0, 200, 7)
    r1 = oracle_mod.transfer(sc, dirs, 2, recv, bounce=True)
    sc2 = S.Scene(**{**sc.arrays(), "albedo": (sc.albedo * 0.5).astype(np.float32)})
    r2 = oracle_mod.transfer(sc2, dirs, 2, recv, bounce=True)
    B1 = r1["T"] - r1["P"][:, None, :]
    B2 = r2["T"] - r2["P"][:, None, :]
    np.testing.assert_allclose(B2, 0.5 * B1, atol=1e-14)
    assert np.max(np.abs(B1)) > 1e-3
    sc0 = S.Scene(**{**sc.arrays(), "albedo": np.zeros_like(sc.albedo)})
    r0 = oracle_mod.transfer(sc0, dirs, 2, recv, bounce=True)
    np.testing.assert_array_equal(r0["T"], np.repeat(r0["P"][:, None, :], 3, axis=1))


# ------------------------------------------------------------------------------------------
# Glossy transfer matrices (Eq. 36-41) and the BRDF pieces of Eq. 15
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("r", [0.1, 0.3, 0.6, 1.0])
def test_ggx_normalised(oracle_mod, r):
    from scipy.integrate import quad

    a = r * r
    val = quad(lambda th: 2 * math.pi * oracle_mod.ggx_D(math.cos(th), a) * math.cos(th) * math.sin(th),
               0, math.pi / 2, epsabs=1e-12, limit=400, points=[min(1e-3, a)])[0]
    assert val == pytest.approx(1.0, abs=1e-7)


def test_fresnel_and_masking_limits(oracle_mod):
    assert oracle_mod.schlick_F(1.0) == pytest.approx(0.04)
    assert oracle_mod.schlick_F(0.0) == pytest.approx(1.0)
    x = np.linspace(1e-4, 1, 50)
    for a in (0.01, 0.3, 1.0):
        g = oracle_mod.smith_G1(x, a)
        assert np.all(g <= 1 + 1e-15) and np.all(g > 0)
        assert oracle_mod.smith_G1(1.0, a) == pytest.approx(1.0)


def test_brdf_kernel_reciprocal_and_white_furnace(oracle_mod):
    rng = np.random.default_rng(5)
    n = np.array([0, 0, 1.0])
    wi = S.unit_vectors(rng, 500)
    wo = S.unit_vectors(rng, 500)
    k1 = oracle_mod.brdf_kernel(n, wi, wo, 0.4, 0.3)
    k2 = oracle_mod.brdf_kernel(n, wo, wi, 0.4, 0.3)
    np.testing.assert_allclose(k1, k2, rtol=1e-12)
    # pure specular part reflects at most all energy: int f_s cos dw_o <= 1
    d = S.direction_set(1 << 16, 1).astype(np.float64)
    for th in (0.1, 0.8, 1.3):
        w_in = np.array([math.sin(th), 0, math.cos(th)])
        ks = oracle_mod.brdf_kernel(n, w_in[None], d, 0.5, 1.0) / math.pi  # m=1 -> f_s only
        alb = 4 * math.pi / d.shape[0] * np.sum(ks * np.maximum(d[:, 2], 0))
        assert 0 < alb <= 1.0


def test_glossy_matrix_structure_rank_one_with_diffuse_kernel(oracle_mod, monkeypatch):
    """With the kernel replaced by the Lambertian indicator, M = P (x) Q exactly, where
    Q_b = sum_o w [n.w_o > 0] Y_b(w_o). Checks the index roles and weights of Eq. 40."""
    sc = S.isotropic_scene(64, 9)
    sc.scales *= 3
    dirs = S.direction_set(128, 3)
    recv = np.arange(0, 64, 9)
    tr = oracle_mod.transfer(sc, dirs, 3, recv)
    monkeypatch.setattr(oracle_mod, "brdf_kernel",
                        lambda n, wi, wo, r, m: ((wo * n).sum(-1) > 0).astype(float) * ((wi * n).sum(-1) > 0))
    M, _ = oracle_mod.glossy(sc, dirs, 3, recv, tr["V"])
    Y = oracle_mod.sh(3, dirs)
    w = 4 * math.pi / 128
    for r, i in enumerate(recv):
        Q = w * ((dirs.astype(float) @ sc.normals[i].astype(float) > 0)[:, None] * Y).sum(0)
        np.testing.assert_allclose(M[r], np.outer(tr["P"][r], Q), atol=1e-13)


# ------------------------------------------------------------------------------------------
# Relight (Eq. 14, Eq. 41)
# ------------------------------------------------------------------------------------------
def test_white_furnace_relight(oracle_mod):
    """Unoccluded Lambertian splat under constant radiance c reflects rho * c."""
    dirs = S.direction_set(1 << 16, 4)
    rng = np.random.default_rng(6)
    nrm = S.unit_vectors(rng, 4)
    sc = _sc([[0, 0, 0], [50, 0, 0], [0, 50, 0], [0, 0, 50]], np.full((4, 3), 0.01), [0.5] * 4, nrm,
             albedo=rng.uniform(0, 1, (4, 3)))
    P = oracle_mod.transfer(sc, dirs, 2, np.arange(4))["P"]
    c = np.array([0.7, 1.1, 1.4])
    L = np.zeros((1, 3, 9))
    L[0, :, 0] = 2 * math.sqrt(math.pi) * c
    col = oracle_mod.relight(P, sc.albedo, L)
    np.testing.assert_allclose(col[0], sc.albedo * c[None, :], rtol=2e-4)


def test_glossy_relight_reduces_to_diffuse_for_rank_one(oracle_mod):
    rng = np.random.default_rng(8)
    P = rng.standard_normal((5, 16))
    Q = rng.standard_normal(16)
    M = P[:, :, None] * Q[None, None, :]
    means = rng.standard_normal((5, 3))
    cam = np.array([3.0, -2.0, 1.0])
    L = rng.standard_normal((2, 3, 16))
    alb = rng.uniform(0, 1, (5, 3))
    v = cam[None] - means
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    s = oracle_mod.sh(3, v) @ Q
    col = oracle_mod.relight(np.zeros((5, 16)), alb, L, glossy_ids=np.arange(5), M=M, means=means, cam_pos=cam,
                             order=3)
    ref = oracle_mod.relight(P * s[:, None], alb, L)
    np.testing.assert_allclose(col, ref, rtol=1e-12, atol=1e-14)


# ------------------------------------------------------------------------------------------
# Morton codes and the radix tree (Sec. 4.4 BVH)
# ------------------------------------------------------------------------------------------
def _decode(code):
    q = [0, 0, 0]
    for b in range(10):
        q[0] |= ((code >> (3 * b + 2)) & 1) << b
        q[1] |= ((code >> (3 * b + 1)) & 1) << b
        q[2] |= ((code >> (3 * b)) & 1) << b
    return q


def test_morton_quantisation_float32(oracle_mod):
    sc = S.isotropic_scene(3000, 12)
    out = oracle_mod.morton_lbvh(sc.means)
    m = sc.means
    lo, hi = m.min(0), m.max(0)
    scale = np.float32(1024) / (hi - lo)  # numpy float32: IEEE single, no contraction
    q = np.clip(np.floor((m - lo) * scale), 0, 1023).astype(int)
    dec = np.array([_decode(int(c)) for c in out["codes"]])
    np.testing.assert_array_equal(dec, q)


def _check_radix_tree(keys, children, root, lo, hi, order):
    """Leaves of each node are the contiguous sorted range, split at the highest differing bit."""
    stack = [(root, lo, hi)]
    seen = []
    while stack:
        node, a, b = stack.pop()
        if node < 0:
            assert a == b and order[a] == -1 - node
            seen.append(a)
            continue
        bit = 63 - (int(keys[a]) ^ int(keys[b])).bit_length() + 1
        mask = 1 << (63 - bit)
        # the split is where that bit flips from 0 to 1
        split = next(p for p in range(a, b) if (int(keys[p + 1]) & mask))
        assert all((int(keys[p]) & mask) == 0 for p in range(a, split + 1))
        l, r = children[node]
        stack.append((l, a, split))
        stack.append((r, split + 1, b))
    assert sorted(seen) == list(range(lo, hi + 1))


def test_radix_tree_definition(oracle_mod):
    sc = S.isotropic_scene(700, 13)
    out = oracle_mod.morton_lbvh(sc.means)
    assert np.all(np.diff(out["keys"].astype(np.uint64)) > 0)
    _check_radix_tree(out["keys"], out["children"], out["roots"][0], 0, 699, out["order"])
    # key low bits are the Gaussian index
    np.testing.assert_array_equal(out["keys"] & np.uint64((1 << 27) - 1), out["order"].astype(np.uint64))


def test_radix_tree_batched_roots(oracle_mod):
    parts = [S.isotropic_scene(n, 50 + n) for n in (5, 1, 40, 17)]
    sc, offs = S.concat_scenes(parts)
    out = oracle_mod.morton_lbvh(sc.means, offs)
    pos = 0
    for b, p in enumerate(parts):
        _check_radix_tree(out["keys"], out["children"], out["roots"][b], pos, pos + p.n - 1, out["order"])
        assert set(out["order"][pos:pos + p.n]) == set(range(offs[b], offs[b + 1]))
        pos += p.n


# ------------------------------------------------------------------------------------------
# Differentiable transfer (gradient oracle of the transfer backward)
# ------------------------------------------------------------------------------------------
def _crowd(n, seed):
    sc = S.surface_scene(n, seed)
    sc.means *= 0.25  # crowd them so that rays meet many occluders
    sc.scales *= 1.5
    return sc


def test_torch_transfer_equals_c_oracle(oracle_mod):
    import torch

    from oracle import transfer_torch as TT

    sc = _crowd(60, 3)
    dirs = S.direction_set(48, 2)
    ref = oracle_mod.transfer(sc, dirs, 3, np.arange(sc.n), t_min=0.0)
    t = lambda a: torch.as_tensor(np.asarray(a, np.float64))
    P = TT.transfer_P(t(sc.means), t(sc.scales), t(sc.quats), t(sc.opacity), t(sc.normals), dirs,
                      oracle_mod.sh(3, dirs)).numpy()
    np.testing.assert_allclose(P, ref["P"], atol=1e-12)
    assert ref["hits"].mean() > 3
    # a receiver subset gives the same rows (every Gaussian still occludes)
    recv = np.array([7, 0, 59, 31])
    Ps = TT.transfer_P(t(sc.means), t(sc.scales), t(sc.quats), t(sc.opacity), t(sc.normals), dirs,
                       oracle_mod.sh(3, dirs), recv=recv).numpy()
    np.testing.assert_allclose(Ps, ref["P"][recv], atol=1e-12)


def test_torch_transfer_autograd_matches_central_differences(oracle_mod):
    import torch

    from oracle import transfer_torch as TT

    sc = _crowd(40, 4)
    dirs = S.direction_set(32, 3)
    Y = oracle_mod.sh(2, dirs)
    rng = np.random.default_rng(9)
    wP = torch.as_tensor(rng.standard_normal((sc.n, 9)))
    ps = [torch.tensor(np.asarray(getattr(sc, f), np.float64), requires_grad=True)
          for f in ("means", "scales", "quats", "opacity", "normals")]

    def f(p):
        return (TT.transfer_P(*p, dirs, Y) * wP).sum()

    grads = torch.autograd.grad(f(ps), ps)
    h = 1e-7
    checked = 0
    for pi, p in enumerate(ps):
        for k in rng.choice(p.numel(), size=6, replace=False):
            pp = [q.detach().clone() for q in ps]
            pm = [q.detach().clone() for q in ps]
            pp[pi].reshape(-1)[k] += h
            pm[pi].reshape(-1)[k] -= h
            with torch.no_grad():
                fd = (f(pp) - f(pm)).item() / (2 * h)
            g = grads[pi].reshape(-1)[k].item()
            assert abs(fd - g) <= 1e-5 * max(1.0, abs(fd)), (pi, k, fd, g)
            checked += 1
    assert checked == 30
    assert float(grads[3].abs().sum()) > 0  # opacity matters


# ---- n-bounce self-transfer (Eq. 34-35) -----------------------------------------------------
def test_multi_bounce_one_bounce_is_eq33(oracle_mod):
    """One bounce of the recursion is the one-bounce transfer T (and its allowance)."""
    sc = _crowd(120, 8)
    dirs = S.direction_set(48, 4)
    tr = oracle_mod.transfer(sc, dirs, 2, np.arange(sc.n), bounce=True)
    T1, a1 = oracle_mod.multi_bounce(sc, dirs, 2, tr, 1)
    np.testing.assert_allclose(T1, tr["T"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(a1, tr["allow_T"], rtol=1e-12, atol=1e-15)
    assert (tr["idx"] >= 0).sum() > 100


class _TwoSplats:
    def __init__(self, normals, albedo):
        self.normals = np.asarray(normals, np.float64)
        self.albedo = np.asarray(albedo, np.float64)


@pytest.mark.parametrize("n", [1, 2, 3, 6])
def test_multi_bounce_two_facing_splats_closed_form(oracle_mod, n):
    """Two splats whose one ray each hits the other: the bounces alternate, so with
    a = w c_A rho_B / pi and b = w c_B rho_A / pi (per channel)
    T_A = P_A sum_{m <= n/2} (ab)^m + a P_B sum_{m <= (n-1)/2} (ab)^m."""
    dirs = np.array([[0, 0, 1.0], [0, 0, -1.0], [1.0, 0, 0], [0, 1.0, 0]])
    nA, nB = np.array([0.0, 0.6, 0.8]), np.array([0.0, 0.28, -0.96])
    sc = _TwoSplats([nA, nB], [[0.9, 0.5, 0.2], [0.3, 0.7, 0.6]])
    rng = np.random.default_rng(3)
    P = rng.standard_normal((2, 9))
    idx = -np.ones((2, 4), np.int64)
    idx[0, 0] = 1  # A's ray along +z hits B
    idx[1, 1] = 0  # B's ray along -z hits A
    tr = dict(P=P, allow_P=np.zeros(2), idx=idx, flags=np.zeros((2, 4), np.int32))
    T, _ = oracle_mod.multi_bounce(sc, dirs, 2, tr, n)
    w = 4 * math.pi / 4
    a = w * max(nA @ dirs[0], 0) * sc.albedo[1] / math.pi
    b = w * max(nB @ dirs[1], 0) * sc.albedo[0] / math.pi
    geo_even = sum((a * b) ** m for m in range(n // 2 + 1))
    geo_odd = sum((a * b) ** m for m in range((n - 1) // 2 + 1))
    TA = geo_even[:, None] * P[0][None, :] + (a * geo_odd)[:, None] * P[1][None, :]
    TB = geo_even[:, None] * P[1][None, :] + (b * geo_odd)[:, None] * P[0][None, :]
    np.testing.assert_allclose(T[0], TA, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(T[1], TB, rtol=1e-13, atol=1e-14)


def test_multi_bounce_converges_to_the_resolvent(oracle_mod):
    """With every bounce kept, T = sum_k W^k P = (I - W)^{-1} P per channel, W[i,j] the summed
    weights w (n_i.w_s)^+ rho_j / pi of receiver i's rays whose index is j."""
    rng = np.random.default_rng(5)
    N, Sd, C = 40, 24, 4
    dirs = S.direction_set(Sd, 6)
    normals = rng.standard_normal((N, 3))
    normals /= np.linalg.norm(normals, axis=1, keepdims=True)
    sc = _TwoSplats(normals, rng.uniform(0.1, 0.6, (N, 3)))
    idx = rng.integers(-N // 2, N, (N, Sd))
    idx[idx < 0] = -1
    P = rng.standard_normal((N, C))
    tr = dict(P=P, allow_P=np.zeros(N), idx=idx, flags=np.zeros((N, Sd), np.int32))
    T, _ = oracle_mod.multi_bounce(sc, dirs, 1, tr, 80)
    w = 4 * math.pi / Sd
    cosw = np.maximum(normals @ dirs.T, 0)
    for ch in range(3):
        W = np.zeros((N, N))
        for i in range(N):
            for s_ in range(Sd):
                if idx[i, s_] >= 0:
                    W[i, idx[i, s_]] += w * cosw[i, s_] * sc.albedo[idx[i, s_], ch] / math.pi
        assert np.max(np.abs(np.linalg.eigvals(W))) < 0.7
        np.testing.assert_allclose(T[:, ch, :], np.linalg.solve(np.eye(N) - W, P), rtol=1e-10, atol=1e-10)


def test_live_hits_stop_at_the_visibility_cut_off(oracle_mod):
    """A ray straight up through a column of m identical occluders hit at their centres
    (alpha = opacity each) takes min(m, q) hits before its transmittance falls below t_min,
    q the first count with (1 - alpha)^q < t_min; all m hits are counted otherwise."""
    m, op = 40, 0.6
    means = [[0, 0, 0]] + [[0, 0, 1.0 + k] for k in range(m)]
    sc = _sc(means, np.full((m + 1, 3), 0.05), [0.5] + [op] * m, np.tile([0, 0, 1.0], (m + 1, 1)))
    dirs = np.array([[0, 0, 1.0]], np.float32)
    for t_min, expect in ((2.0 ** -30, int(np.ceil(np.log(2.0 ** -30) / np.log(1 - op)))), (0.0, m)):
        tr = oracle_mod.trace(sc, dirs, 1, [0], t_min=t_min)
        assert tr["hits"][0] == m
        assert tr["hits_live"][0] == min(m, expect), (t_min, tr["hits_live"][0])
    assert int(np.ceil(np.log(2.0 ** -30) / np.log(1 - op))) < m  # the cut-off is inside the column


def test_multi_bounce_allowance_covers_switching_a_flagged_ray(oracle_mod):
    """For a ray flagged rounding-ambiguous, taking any of its other candidates changes the
    n-bounce T by no more than the carried allowance."""
    rng = np.random.default_rng(11)
    N, Sd, C = 12, 8, 4
    dirs = S.direction_set(Sd, 3)
    normals = rng.standard_normal((N, 3))
    normals /= np.linalg.norm(normals, axis=1, keepdims=True)
    sc = _TwoSplats(normals, rng.uniform(0.1, 0.9, (N, 3)))
    idx = rng.integers(-2, N, (N, Sd))
    idx[idx < 0] = -1
    flags = np.zeros((N, Sd), np.int32)
    cand = -np.ones((N, Sd, 4), np.int64)
    amb = [(0, 1), (3, 2), (5, 0)]
    for i, s_ in amb:
        flags[i, s_] = oracle_mod.RF_AMBIG_ARGMAX
        cand[i, s_, :3] = rng.integers(0, N, 3)
    P = rng.standard_normal((N, C))
    tr = dict(P=P, allow_P=np.zeros(N), idx=idx, flags=flags, cand=cand)
    for nb in (1, 3):
        T, allow = oracle_mod.multi_bounce(sc, dirs, 1, tr, nb)
        for i, s_ in amb:
            for alt in list(cand[i, s_, :3]) + [-1]:
                idx2 = idx.copy()
                idx2[i, s_] = alt
                T2, _ = oracle_mod.multi_bounce(sc, dirs, 1, dict(tr, idx=idx2, flags=np.zeros_like(flags)), nb)
                # a single switch moves receiver i directly and, through later bounces, others
                assert np.all(np.linalg.norm(T2 - T, axis=2)[i] <= allow[i] + 1e-12), (nb, i, alt)


@pytest.mark.parametrize("nb", [1, 3])
def test_torch_bounce_equals_the_recursion_and_central_differences(oracle_mod, nb):
    """The differentiable bounce restatement equals the numpy recursion (itself pinned to Eq. 33
    and the closed forms above) on a traced index matrix, and its autograd gradients with respect
    to P, albedo and normals equal central differences."""
    import torch

    from oracle import transfer_torch as TT

    sc = _crowd(90, 12)
    dirs = S.direction_set(40, 5)
    tr = oracle_mod.transfer(sc, dirs, 2, np.arange(sc.n), bounce=True)
    Tref, _ = oracle_mod.multi_bounce(sc, dirs, 2, tr, nb)
    t = lambda a, rg=False: torch.tensor(np.asarray(a, np.float64), requires_grad=rg)
    P, rho, nrm = t(tr["P"], True), t(sc.albedo, True), t(sc.normals, True)
    T = TT.bounce_T(P, tr["idx"], dirs, nrm, rho, nb)
    np.testing.assert_allclose(T.detach().numpy(), Tref, rtol=0, atol=1e-12)
    assert (tr["idx"] >= 0).sum() > 100
    rng = np.random.default_rng(nb)
    W = torch.as_tensor(rng.standard_normal(tuple(T.shape)))
    f = lambda p, r, n: (TT.bounce_T(p, tr["idx"], dirs, n, r, nb) * W).sum()
    grads = torch.autograd.grad(f(P, rho, nrm), (P, rho, nrm))
    h = 1e-7
    for gi, base in enumerate((P, rho, nrm)):
        for k in rng.choice(base.numel(), size=8, replace=False):
            args_p = [q.detach().clone() for q in (P, rho, nrm)]
            args_m = [q.detach().clone() for q in (P, rho, nrm)]
            args_p[gi].reshape(-1)[k] += h
            args_m[gi].reshape(-1)[k] -= h
            with torch.no_grad():
                fd = (f(*args_p) - f(*args_m)).item() / (2 * h)
            g = grads[gi].reshape(-1)[k].item()
            assert abs(fd - g) <= 1e-6 * max(1.0, abs(fd)), (gi, k, fd, g)
    assert all(float(g.abs().sum()) > 0 for g in grads)


def test_torch_glossy_equals_numpy_and_central_differences(oracle_mod):
    """The differentiable glossy matrices (Eq. 40) equal the numpy form (pinned above by the GGX
    normalisation, reciprocity and the rank-one structure) on traced visibilities, and their
    autograd gradients with respect to V, the normal, roughness and metallic equal central
    differences."""
    import torch

    from oracle import transfer_torch as TT

    sc = _crowd(60, 21)
    rng = np.random.default_rng(21)
    sc.roughness = rng.uniform(0.3, 0.9, sc.n)
    sc.metallic = rng.uniform(0.0, 1.0, sc.n)
    dirs = S.direction_set(24, 7)
    recv = np.array([3, 17, 40])
    tr = oracle_mod.transfer(sc, dirs, 2, recv)
    M_ref, _ = oracle_mod.glossy(sc, dirs, 2, recv, tr["V"])
    Y = oracle_mod.sh(2, dirs)
    t = lambda a: torch.tensor(np.asarray(a, np.float64), requires_grad=True)
    V, nrm, r, m = t(tr["V"]), t(sc.normals[recv]), t(sc.roughness[recv]), t(sc.metallic[recv])
    M = TT.glossy_M(V, nrm, r, m, dirs, Y)
    np.testing.assert_allclose(M.detach().numpy(), M_ref, rtol=0, atol=1e-12 * max(1.0, np.abs(M_ref).max()))
    W = torch.as_tensor(rng.standard_normal(tuple(M.shape)))
    f = lambda *a: (TT.glossy_M(*a, dirs, Y) * W).sum()
    args = (V, nrm, r, m)
    grads = torch.autograd.grad(f(*args), args)
    h = 1e-7
    for gi, base in enumerate(args):
        for k in rng.choice(base.numel(), size=min(6, base.numel()), replace=False):
            ap = [q.detach().clone() for q in args]
            am = [q.detach().clone() for q in args]
            ap[gi].reshape(-1)[k] += h
            am[gi].reshape(-1)[k] -= h
            with torch.no_grad():
                fd = (f(*ap) - f(*am)).item() / (2 * h)
            g = grads[gi].reshape(-1)[k].item()
            assert abs(fd - g) <= 2e-6 * max(1.0, abs(fd)), (gi, k, fd, g)
    assert all(float(g.abs().sum()) > 0 for g in grads)
