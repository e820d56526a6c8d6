"""GPU parity of the BVH build and the transfer precompute against the FP64 oracle.

Tolerances (norm-wise per receiver, see oracle.transfer for the allowance):
  ||P_gpu - P_ref|| <= 1e-4 * max(||P_ref||, 1e-3 * ||P_unoccluded||) + allow_P
  ||T_gpu - T_ref|| likewise over the three channels, with the root-sum-square of the
  per-channel allowances (each bounds the change of one channel's C-vector; a flipped
  visibility decision moves P, and so every channel of T = P + bounce, at once)
Integer outputs (Morton keys, sorted order, tree topology, index matrix on unflagged rays)
are compared bit-exactly.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2408_03538_gb300 import api, scenes as S

pytestmark = pytest.mark.gpu
TOL = 1e-4


def _gt(scene):
    return api.GaussianTensors.from_scene(scene)


def _offsets(sizes):
    o = np.zeros(len(sizes) + 1, np.int64)
    o[1:] = np.cumsum(sizes)
    return torch.from_numpy(o).cuda()


def _children_as_ids(children, order):
    ch = children.copy()
    leaf = ch < 0
    ch[leaf] = -1 - order[~ch[leaf]]
    return ch


@pytest.mark.parametrize("sizes", [[1024], [1000], [2], [1], [5, 1, 40, 17], [300, 0, 299]])
def test_bvh_bit_exact(sizes):
    parts = [S.isotropic_scene(n, 100 + i + n) for i, n in enumerate(sizes)]
    sc, offs = S.concat_scenes(parts)
    g = _gt(sc)
    st = api.Status()
    bvh = api.build_bvh(g, torch.from_numpy(offs).cuda(), st)
    torch.cuda.synchronize()
    assert st.read() == 0
    ref = oracle.morton_lbvh(sc.means, offs)
    n = sc.n
    keys = bvh.view("keys", torch.int64, (n,)).cpu().numpy().view(np.uint64)
    order = bvh.view("order", torch.int32, (n,)).cpu().numpy()
    np.testing.assert_array_equal(keys, ref["keys"])
    np.testing.assert_array_equal(order, ref["order"])
    roots = bvh.view("roots", torch.int32, (len(sizes),)).cpu().numpy()
    if n > 1:
        nodes = bvh.view("nodes", torch.float32, (n - 1, 16)).cpu().numpy()
        ch = nodes[:, 12:14].copy().view(np.int32)
        np.testing.assert_array_equal(_children_as_ids(ch, order), ref["children"])
        # every child box contains the exact FP64 3-sigma box of its subtree
        box = oracle.aabb_3sigma(sc)
        sub = np.zeros((2 * n - 1, 6))
        lo_hi = {}

        def subtree_box(c):
            if c < 0:
                return box[order[~c]]
            if c in lo_hi:
                return lo_hi[c]
            a, b = subtree_box(int(ch[c, 0])), subtree_box(int(ch[c, 1]))
            lo_hi[c] = np.concatenate([np.minimum(a[:3], b[:3]), np.maximum(a[3:], b[3:])])
            return lo_hi[c]

        import sys
        sys.setrecursionlimit(10000)
        for node in range(n - 1):
            for slot in range(2):
                bx = nodes[node, 6 * slot:6 * slot + 6].astype(np.float64)
                ex = subtree_box(int(ch[node, slot]))
                assert np.all(bx[:3] <= ex[:3]) and np.all(bx[3:] >= ex[3:])
    for b, r in enumerate(ref["roots"]):
        if sizes[b] == 0:
            continue
        rr = roots[b]
        if rr < 0:
            assert -1 - order[~rr] == r
        else:
            assert rr == r


def _transfer_gpu(scene, dirs, order, bounce=False, glossy=False, t_min=api.DEFAULT_T_MIN, walk=0):
    g = _gt(scene)
    st = api.Status()
    bvh = api.build_bvh(g, status=st)
    d = torch.from_numpy(dirs).cuda()
    out = api.precompute_transfer(g, bvh, d, order, bounce=bounce, glossy=glossy, t_min=t_min, status=st,
                                  walk=walk)
    torch.cuda.synchronize()
    assert st.read() == 0
    return {k: (v.cpu().numpy() if torch.is_tensor(v) else v) for k, v in out.items()}


def _check_norm(gpu, ref, allow, floor, tol=TOL):
    err = np.linalg.norm((gpu - ref).reshape(len(ref), -1), axis=1)
    lim = tol * np.maximum(np.linalg.norm(ref.reshape(len(ref), -1), axis=1), floor) + allow
    bad = np.nonzero(err > lim)[0]
    assert bad.size == 0, f"{bad.size} receivers over tolerance, worst {np.max(err / lim):.3g}x at {bad[:5]}"
    return float(np.max(err / np.maximum(np.linalg.norm(ref.reshape(len(ref), -1), axis=1), floor)))


def test_transfer_shadow_tiny_config_all_receivers():
    """1,024 isotropic Gaussians, order 2, S = 64 (the plain-method tiny workload)."""
    sc = S.make_scene("tiny-1k")
    dirs = S.direction_set(64, S.config_seed(0))
    out = _transfer_gpu(sc, dirs, 2)
    ref = oracle.transfer(sc, dirs, 2, np.arange(sc.n))
    floor = 1e-3 * oracle.unoccluded_norm(2)
    _check_norm(out["P"], ref["P"], ref["allow_P"], floor)
    assert np.mean(ref["hits"] / np.maximum(ref["traced"], 1)) > 5  # the workload really occludes


def test_transfer_exact_without_early_exit_and_unshadowed():
    sc = S.isotropic_scene(700, 5)
    dirs = S.direction_set(96, 3)
    out = _transfer_gpu(sc, dirs, 3, t_min=0.0)
    ref = oracle.transfer(sc, dirs, 3, np.arange(sc.n), t_min=0.0)
    _check_norm(out["P"], ref["P"], ref["allow_P"], 1e-3 * oracle.unoccluded_norm(3))
    # without shadowing every receiver gets the discrete clamped-cosine projection
    g = _gt(sc)
    bvh = api.build_bvh(g)
    P = api.precompute_transfer(g, bvh, torch.from_numpy(dirs).cuda(), 3, shadow=False)["P"].cpu().numpy()
    refu = oracle.transfer(sc, dirs, 3, np.arange(sc.n), shadow=False)["P"]
    np.testing.assert_allclose(P, refu, atol=2e-6, rtol=0)


@pytest.mark.parametrize("n,order,nd", [(1, 2, 64), (2, 1, 32), (3, 3, 1), (33, 3, 100)])
def test_transfer_edge_sizes(n, order, nd):
    sc = S_mod_scene(n)
    dirs = S_dirs(nd)
    out = _transfer_gpu(sc, dirs, order, bounce=True)
    ref = oracle.transfer(sc, dirs, order, np.arange(sc.n), bounce=True)
    _check_norm(out["P"], ref["P"], ref["allow_P"], 1e-3 * oracle.unoccluded_norm(order))
    _check_norm(out["T"], ref["T"], np.linalg.norm(ref["allow_T"], axis=1), 1e-3 * oracle.unoccluded_norm(order))


def S_mod_scene(n):
    sc = S.isotropic_scene(n, 900 + n)
    sc.means *= 0.2  # crowd them so that they occlude each other
    return sc


def S_dirs(k):
    return S.direction_set(k, 17)


def test_transfer_bounce_surface_scene():
    """Anisotropic surface splats, order 3, S = 128, shadow + one bounce, every receiver."""
    sc = S.surface_scene(3000, S.config_seed(1))
    dirs = S.direction_set(128, S.config_seed(1))
    out = _transfer_gpu(sc, dirs, 3, bounce=True)
    ref = oracle.transfer(sc, dirs, 3, np.arange(sc.n), bounce=True)
    floor = 1e-3 * oracle.unoccluded_norm(3)
    _check_norm(out["P"], ref["P"], ref["allow_P"], floor)
    _check_norm(out["T"], ref["T"], np.linalg.norm(ref["allow_T"], axis=1), floor)
    # index matrix: exact on every ray without a flagged decision
    clean = (ref["flags"] & (oracle.RF_AMBIG_HIT | oracle.RF_AMBIG_ARGMAX)) == 0
    np.testing.assert_array_equal(out["idx"][clean], ref["idx"][clean])
    assert clean.mean() > 0.99
    assert np.mean(ref["idx"] >= 0) > 0.05  # the bounce term is exercised


@pytest.mark.parametrize("t_min", [0.0, 1e-3])
def test_transfer_bounce_cutoff_variants(t_min):
    """Index matrix and bounce without the early cut-off (t_min = 0, the literal argmax) and
    with a coarse one (t_min = 1e-3): both sides apply the same candidate rule."""
    sc = S.surface_scene(1200, 33)
    dirs = S.direction_set(64, 9)
    out = _transfer_gpu(sc, dirs, 2, bounce=True, t_min=t_min)
    ref = oracle.transfer(sc, dirs, 2, np.arange(sc.n), bounce=True, t_min=t_min)
    floor = 1e-3 * oracle.unoccluded_norm(2)
    _check_norm(out["P"], ref["P"], ref["allow_P"], floor)
    _check_norm(out["T"], ref["T"], np.linalg.norm(ref["allow_T"], axis=1), floor)
    clean = (ref["flags"] & (oracle.RF_AMBIG_HIT | oracle.RF_AMBIG_ARGMAX)) == 0
    np.testing.assert_array_equal(out["idx"][clean], ref["idx"][clean])


@pytest.mark.parametrize("kb", [1, 2, 4, 8])
def test_index_buffer_sizes_agree(kb):
    sc = S.surface_scene(2000, 34)
    dirs = torch.from_numpy(S.direction_set(64, 10)).cuda()
    g = _gt(sc)
    bvh = api.build_bvh(g)
    a = api.precompute_transfer(g, bvh, dirs, 2, bounce=True, index_buffer=kb)["idx"].cpu().numpy()
    ref = oracle.transfer(sc, dirs.cpu().numpy(), 2, np.arange(sc.n), bounce=True)
    clean = (ref["flags"] & (oracle.RF_AMBIG_HIT | oracle.RF_AMBIG_ARGMAX)) == 0
    np.testing.assert_array_equal(a[clean], ref["idx"][clean])


def test_transfer_full_size_sampled_receivers():
    """The 100k-Gaussian surface workload (order 3, S = 256, shadow + bounce) on the GPU,
    checked on seeded sampled receivers that the oracle computes one by one."""
    sc = S.make_scene("surface-100k")
    dirs = S.direction_set(256, S.config_seed(1))
    out = _transfer_gpu(sc, dirs, 3, bounce=True)
    rng = np.random.default_rng(4)
    recv = np.sort(rng.choice(sc.n, size=256, replace=False))
    ref = oracle.transfer(sc, dirs, 3, recv, bounce=True, bounce_T=False)
    floor = 1e-3 * oracle.unoccluded_norm(3)
    _check_norm(out["P"][recv], ref["P"], ref["allow_P"], floor)
    clean = (ref["flags"] & (oracle.RF_AMBIG_HIT | oracle.RF_AMBIG_ARGMAX)) == 0
    np.testing.assert_array_equal(out["idx"][recv][clean], ref["idx"][clean])
    # T (Eq. 33) needs P of every splat the index matrix points to: a subset of the receivers
    sub_r = recv[::16]
    refT = oracle.transfer(sc, dirs, 3, sub_r, bounce=True)
    _check_norm(out["T"][sub_r], refT["T"], np.linalg.norm(refT["allow_T"], axis=1), floor)
    # properties that hold everywhere: finite, idx in range, untraced rays have no index
    assert np.all(np.isfinite(out["T"]))
    assert out["idx"].min() >= -1 and out["idx"].max() < sc.n
    c = sc.normals.astype(np.float64) @ dirs.astype(np.float64).T
    assert np.all(out["idx"][c <= 0] == -1)


def test_glossy_matrices():
    sc = S.surface_scene(1500, 77)
    rng = np.random.default_rng(5)
    sc.glossy_mask = (rng.random(sc.n) < 0.3).astype(np.uint8)
    sc.roughness = rng.uniform(0.1, 0.6, sc.n).astype(np.float32)
    sc.metallic = rng.uniform(0.0, 1.0, sc.n).astype(np.float32)
    dirs = S.direction_set(64, 8)
    out = _transfer_gpu(sc, dirs, 3, glossy=True)
    gids = np.nonzero(sc.glossy_mask)[0]
    assert out["n_glossy"] == gids.size
    tr = oracle.transfer(sc, dirs, 3, gids)
    Vallow = tr["dV"] + np.where((tr["flags"] & oracle.RF_TRACED) != 0, api.DEFAULT_T_MIN, 0.0)
    M, allow = oracle.glossy(sc, dirs, 3, gids, tr["V"], Vallow)
    floor = 1e-3 * np.median(np.linalg.norm(M.reshape(len(M), -1), axis=1))
    _check_norm(out["M"], M, allow, floor)


# ---- transfer backward (gradients of P through the recomputed walks) ----------------------
_GRAD_FIELDS = ("means", "scales", "quats", "opacity", "normals")


def _crowded(n, seed, f=0.4):
    sc = S.surface_scene(n, seed)
    sc.means *= f
    sc.scales *= 1.5
    return sc


def _transfer_grads(sc, dirs, order, wP, shadow=True, t_min=0.0):
    """(GPU gradients, FP64 autograd gradients) of L = sum(wP * P)."""
    from oracle import transfer_torch as TT

    g = _gt(sc)
    st = api.Status()
    bvh = api.build_bvh(g, status=st)
    d = torch.from_numpy(dirs).cuda()
    out = api.precompute_transfer_backward(g, bvh, d, order, torch.from_numpy(wP).cuda(), shadow=shadow,
                                           t_min=t_min, status=st)
    torch.cuda.synchronize()
    assert st.read() == 0
    gpu = {f: out["d_" + f].cpu().numpy().astype(np.float64) for f in _GRAD_FIELDS}
    ps = [torch.tensor(np.asarray(getattr(sc, f), np.float64), requires_grad=True) for f in _GRAD_FIELDS]
    Y = oracle.sh(order, dirs)
    if shadow:
        P = TT.transfer_P(*ps, dirs, Y)
    else:  # unshadowed: V = 1, only the cosine depends on the Gaussians
        dd = torch.as_tensor(np.asarray(dirs, np.float64))
        c = ps[4] @ dd.T
        P = torch.where((c > 0).detach(), 4.0 * math.pi / len(dirs) * c, torch.zeros_like(c)) @ torch.as_tensor(Y)
    ref = torch.autograd.grad((P * torch.as_tensor(wP.astype(np.float64))).sum(), ps, allow_unused=True)
    ref = {f: (r.numpy() if r is not None else np.zeros(getattr(sc, f).shape)) for f, r in zip(_GRAD_FIELDS, ref)}
    return gpu, ref


def _check_grads(gpu, ref, tol=2e-3):
    """Norm-wise and element-wise per field; a field whose exact gradient vanishes (the rotation
    of an isotropic Gaussian) is held to the FP32 residue, 1e-3 of the largest field's scale."""
    top = max(np.linalg.norm(ref[f]) for f in _GRAD_FIELDS)
    top_el = max(np.abs(ref[f]).max() for f in _GRAD_FIELDS)
    for f in _GRAD_FIELDS:
        a, b = gpu[f].ravel(), ref[f].ravel()
        nb = max(np.linalg.norm(b), 1e-3 * top)
        assert np.linalg.norm(a - b) <= tol * nb, (f, np.linalg.norm(a - b) / nb)
        # element-wise: every entry within tol of the field's largest entry
        np.testing.assert_allclose(a, b, rtol=0, atol=tol * max(np.abs(b).max(), 1e-3 * top_el), err_msg=f)


@pytest.mark.parametrize("n,order,nd,t_min", [(300, 3, 64, 0.0), (600, 2, 48, api.DEFAULT_T_MIN), (257, 1, 33, 0.0),
                                               (280, 5, 48, 0.0), (200, 6, 40, api.DEFAULT_T_MIN)])
def test_transfer_backward_matches_autograd(n, order, nd, t_min):
    """dL/d(Gaussians) for L = sum(wP * P) against FP64 autograd through the brute-force P."""
    sc = _crowded(n, 11 + n)
    dirs = S.direction_set(nd, 5)
    wP = np.random.default_rng(n).standard_normal((sc.n, (order + 1) ** 2)).astype(np.float32)
    gpu, ref = _transfer_grads(sc, dirs, order, wP, t_min=t_min)
    _check_grads(gpu, ref)
    assert np.abs(ref["opacity"]).sum() > 0 and np.abs(ref["means"]).sum() > 0


def test_transfer_backward_unshadowed_and_tiny():
    sc = _crowded(200, 3)
    dirs = S.direction_set(64, 1)
    wP = np.random.default_rng(1).standard_normal((sc.n, 16)).astype(np.float32)
    gpu, ref = _transfer_grads(sc, dirs, 3, wP, shadow=False)
    _check_grads(gpu, ref)
    for f in ("means", "scales", "quats", "opacity"):
        assert not gpu[f].any()
    # a lone Gaussian has no occluders; two Gaussians shadow each other at most
    for n in (1, 2):
        sc = _crowded(n, 4, f=0.01)
        gpu, ref = _transfer_grads(sc, dirs, 3, wP[:n])
        _check_grads(gpu, ref)


def test_transfer_backward_full_size_sampled_receivers():
    """diff-300k (300,000 isotropic Gaussians in [-1,1]^3, order 3, S = 128): dP is non-zero on
    64 receivers next to the faces of the cube with their normals facing out (inside it a ray's
    visibility is ~1e-120, so there is no gradient to check), so the GPU gradient over all
    300,000 Gaussians is exactly theirs; FP64 autograd through the brute-force P gives the
    reference."""
    from oracle import transfer_torch as TT

    sc = S.make_scene("diff-300k")
    dirs = S.direction_set(128, S.config_seed(3))
    order = 3
    rng = np.random.default_rng(21)
    m = np.asarray(sc.means, np.float64)
    face = np.argmax(np.abs(m), axis=1)
    ar = np.arange(sc.n)
    outward = np.asarray(sc.normals, np.float64)[ar, face] * np.sign(m[ar, face])
    near_face = np.nonzero((np.abs(m[ar, face]) > 0.99) & (outward > 0.7))[0]
    recv = np.sort(rng.choice(near_face, size=64, replace=False))
    wP = np.zeros((sc.n, 16), np.float32)
    wP[recv] = rng.standard_normal((recv.size, 16))
    g = _gt(sc)
    st = api.Status()
    bvh = api.build_bvh(g, status=st)
    out = api.precompute_transfer_backward(g, bvh, torch.from_numpy(dirs).cuda(), order,
                                           torch.from_numpy(wP).cuda(), status=st)
    torch.cuda.synchronize()
    assert st.read() == 0
    gpu = {f: out["d_" + f].cpu().numpy().astype(np.float64) for f in _GRAD_FIELDS}
    ps = [torch.tensor(np.asarray(getattr(sc, f), np.float64), requires_grad=True) for f in _GRAD_FIELDS]
    Y = oracle.sh(order, dirs)
    P = TT.transfer_P(*ps, dirs, Y, recv=recv)
    (P * torch.as_tensor(wP[recv].astype(np.float64))).sum().backward()
    ref = {f: p.grad.numpy() for f, p in zip(_GRAD_FIELDS, ps)}
    _check_grads(gpu, ref)
    assert np.count_nonzero(ref["opacity"]) > 100


def test_tiled_1m_glossy_full_size_sampled():
    """1,000,000 Gaussians (the surface scene tiled 5 x 2 with a random rotation per instance,
    30 % glossy), order 3, S = 256, shadow + bounce + glossy in one call: sampled diffuse and
    glossy receivers against the oracle (P, T, the index matrix, the 16 x 16 matrices M)."""
    sc = S.make_scene("tiled-1m-glossy")
    dirs = S.direction_set(256, S.config_seed(2))
    out = _transfer_gpu(sc, dirs, 3, bounce=True, glossy=True)
    rng = np.random.default_rng(12)
    gl = np.nonzero(sc.glossy_mask)[0]
    assert out["n_glossy"] == gl.size
    recv = np.sort(np.concatenate([rng.choice(np.nonzero(sc.glossy_mask == 0)[0], 192, replace=False),
                                   rng.choice(gl, 64, replace=False)]))
    ref = oracle.transfer(sc, dirs, 3, recv, bounce=True, bounce_T=False)
    floor = 1e-3 * oracle.unoccluded_norm(3)
    _check_norm(out["P"][recv], ref["P"], ref["allow_P"], floor)
    clean = (ref["flags"] & (oracle.RF_AMBIG_HIT | oracle.RF_AMBIG_ARGMAX)) == 0
    np.testing.assert_array_equal(out["idx"][recv][clean], ref["idx"][clean])
    sub_r = recv[::32]  # T needs P of every index target: a subset
    refT = oracle.transfer(sc, dirs, 3, sub_r, bounce=True)
    _check_norm(out["T"][sub_r], refT["T"], np.linalg.norm(refT["allow_T"], axis=1), floor)
    g_recv = recv[sc.glossy_mask[recv] != 0]
    rows = np.searchsorted(gl, g_recv)
    sel = np.isin(recv, g_recv)
    Vallow = ref["dV"][sel] + np.where((ref["flags"][sel] & oracle.RF_TRACED) != 0, api.DEFAULT_T_MIN, 0.0)
    M, allow = oracle.glossy(sc, dirs, 3, g_recv, ref["V"][sel], Vallow)
    _check_norm(out["M"][rows], M, allow, 1e-3 * np.median(np.linalg.norm(M.reshape(len(M), -1), axis=1)))
    assert np.all(np.isfinite(out["M"])) and np.all(np.isfinite(out["T"]))


def test_walks_differ_only_inside_rounding_bands_full_size():
    """The packet walk (a planar test per packet) and the per-ray walk take their hit decisions
    in different FP32 arithmetic. At full size (1M Gaussians, S = 256, shadow + bounce) they
    agree on almost every ray; on the receivers where they differ most, both lie within the
    oracle's allowance and match its index matrix on every unflagged ray."""
    sc = S.make_scene("tiled-1m-glossy")
    dirs = S.direction_set(256, S.config_seed(2))
    o0 = _transfer_gpu(sc, dirs, 3, bounce=True, walk=0)
    o1 = _transfer_gpu(sc, dirs, 3, bounce=True, walk=1)
    dP = np.linalg.norm(o0["P"] - o1["P"], axis=1)
    didx = (o0["idx"] != o1["idx"]).sum(axis=1)
    assert np.mean(o0["idx"] != o1["idx"]) < 1e-3
    worst = np.unique(np.concatenate([np.argsort(dP)[-6:], np.argsort(didx)[-6:]]))
    ref = oracle.transfer(sc, dirs, 3, worst, bounce=True, bounce_T=False)
    floor = 1e-3 * oracle.unoccluded_norm(3)
    clean = (ref["flags"] & (oracle.RF_AMBIG_HIT | oracle.RF_AMBIG_ARGMAX)) == 0
    for o in (o0, o1):
        _check_norm(o["P"][worst], ref["P"], ref["allow_P"], floor)
        np.testing.assert_array_equal(o["idx"][worst][clean], ref["idx"][clean])


# ---- n-bounce self-transfer (Eq. 34-35) -----------------------------------------------------
@pytest.mark.parametrize("nb", [2, 3, 5])
def test_multi_bounce_matches_oracle(nb):
    """T = P + T^1 + ... + T^n over the index matrix, every receiver of a crowded 400-splat
    scene, against the oracle's recursion (norm-wise 1e-4 + the carried allowance)."""
    sc = _crowded(400, 17)
    dirs = S.direction_set(64, 9)
    g = _gt(sc)
    st = api.Status()
    bvh = api.build_bvh(g, status=st)
    T = api.precompute_transfer(g, bvh, torch.from_numpy(dirs).cuda(), 2, bounce=True, n_bounces=nb,
                                status=st)["T"].cpu().numpy()
    torch.cuda.synchronize()
    assert st.read() == 0
    tr = oracle.transfer(sc, dirs, 2, np.arange(sc.n), bounce=True)
    Tref, allow = oracle.multi_bounce(sc, dirs, 2, tr, nb)
    _check_norm(T, Tref, np.linalg.norm(allow, axis=1), 1e-3 * oracle.unoccluded_norm(2))
    # the later bounces matter here: the n-bounce T differs from the one-bounce T
    assert np.linalg.norm(Tref - tr["T"]) > 1e-3 * np.linalg.norm(tr["T"])


def test_multi_bounce_full_size_is_polynomial_in_albedo():
    """At the 100k surface workload size: the index matrix does not depend on albedo, so with
    all albedos scaled by s the bounce part of a two-bounce T is exactly a s + b s^2; three
    scales fix it, a fourth is predicted. One bounce requested explicitly equals the default."""
    sc = S.make_scene("surface-100k")
    dirs = torch.from_numpy(S.direction_set(256, S.config_seed(1))).cuda()
    g = _gt(sc)
    bvh = api.build_bvh(g)
    t1 = api.precompute_transfer(g, bvh, dirs, 3, bounce=True)
    t1b = api.precompute_transfer(g, bvh, dirs, 3, bounce=True, n_bounces=1)
    assert torch.equal(t1["T"], t1b["T"]) and torch.equal(t1["idx"], t1b["idx"])
    P = t1["P"].double()[:, None, :]
    D = {}
    for s_ in (1.0, 0.5, 0.25):
        gs = api.GaussianTensors(g.means, g.scales, g.quats, g.opacity, g.normals, (g.albedo * s_).contiguous())
        out = api.precompute_transfer(gs, bvh, dirs, 3, bounce=True, n_bounces=2)
        assert torch.equal(out["idx"], t1["idx"])
        D[s_] = out["T"].double() - P
    b = 2.0 * (D[1.0] - 2.0 * D[0.5])
    a = D[1.0] - b
    pred = a / 4 + b / 16
    err = (D[0.25] - pred).norm() / D[0.25].norm()
    assert float(err) < 1e-5, float(err)
    assert float(b.norm()) > 1e-3 * float(a.norm())  # the second bounce is there


# ---- SH orders 4-6 (25-49 coefficients): shadowed transfer and FP32 relight -------------------
@pytest.mark.parametrize("order", [4, 6])
def test_high_order_transfer_and_relight_match_oracle(order):
    """Orders above 3 project through a per-call SH table (one lane per coefficient); P against
    the oracle (norm-wise 1e-4 + allowance), and the FP32 relight of seeded scalar and RGB
    transfers at that order against the oracle."""
    sc = S.isotropic_scene(700, 60 + order)
    dirs = S.direction_set(96, 7)
    out = _transfer_gpu(sc, dirs, order)
    ref = oracle.transfer(sc, dirs, order, np.arange(sc.n))
    _check_norm(out["P"], ref["P"], ref["allow_P"], 1e-3 * oracle.unoccluded_norm(order))
    C = (order + 1) ** 2
    rng = np.random.default_rng(order)
    Lsh = rng.standard_normal((5, 3, C)).astype(np.float32)
    for Tin in (rng.standard_normal((sc.n, C)).astype(np.float32),
                rng.standard_normal((sc.n, 3, C)).astype(np.float32)):
        col = api.relight(torch.from_numpy(Tin).cuda(), _gt(sc).albedo, torch.from_numpy(Lsh).cuda(),
                          order).cpu().numpy()
        cref = oracle.relight(Tin, sc.albedo, Lsh)
        err = oracle.norm_err(col.transpose(1, 0, 2), cref.transpose(1, 0, 2), 1e-3)
        assert err.max() < 1e-5


def test_high_order_rejects_what_it_does_not_cover():
    sc = S.isotropic_scene(50, 3)
    sc.glossy_mask[:10] = 1
    g = _gt(sc)
    bvh = api.build_bvh(g)
    d = torch.from_numpy(S.direction_set(32, 1)).cuda()
    with pytest.raises(Exception):  # order 6 glossy matrices of 1024 directions: 614 KB of shared memory
        api.precompute_transfer(g, bvh, torch.from_numpy(S.direction_set(1024, 1)).cuda(), 6, glossy=True)
    with pytest.raises(Exception):
        api.precompute_transfer(g, bvh, d, 7)


@pytest.mark.parametrize("order", [4, 6])
def test_high_order_glossy_matrices(order):
    """The C x C glossy matrices (Eq. 40) at orders 4 and 6 (25 x 25, 49 x 49) against the oracle."""
    sc = S.surface_scene(900, 70 + order)
    rng = np.random.default_rng(order)
    sc.glossy_mask = (rng.random(sc.n) < 0.2).astype(np.uint8)
    sc.roughness = rng.uniform(0.2, 0.8, sc.n).astype(np.float32)
    sc.metallic = rng.uniform(0.0, 1.0, sc.n).astype(np.float32)
    dirs = S.direction_set(64, 8)
    out = _transfer_gpu(sc, dirs, order, glossy=True)
    gids = np.nonzero(sc.glossy_mask)[0]
    assert out["n_glossy"] == gids.size and out["M"].shape[1:] == ((order + 1) ** 2, (order + 1) ** 2)
    tr = oracle.transfer(sc, dirs, order, gids)
    Vallow = tr["dV"] + np.where((tr["flags"] & oracle.RF_TRACED) != 0, api.DEFAULT_T_MIN, 0.0)
    M, allow = oracle.glossy(sc, dirs, order, gids, tr["V"], Vallow)
    floor = 1e-3 * np.median(np.linalg.norm(M.reshape(len(M), -1), axis=1))
    _check_norm(out["M"], M, allow, floor)


@pytest.mark.parametrize("nb", [1, 3])
def test_high_order_bounce_matches_oracle(nb):
    """Order 6 (49 coefficients) with the one- and three-bounce self-transfer against the
    oracle (every receiver of a crowded scene)."""
    sc = _crowded(300, 23)
    dirs = S.direction_set(64, 9)
    g = _gt(sc)
    st = api.Status()
    bvh = api.build_bvh(g, status=st)
    T = api.precompute_transfer(g, bvh, torch.from_numpy(dirs).cuda(), 6, bounce=True, n_bounces=nb,
                                status=st)["T"].cpu().numpy()
    torch.cuda.synchronize()
    assert st.read() == 0
    tr = oracle.transfer(sc, dirs, 6, np.arange(sc.n), bounce=True)
    Tref, allow = oracle.multi_bounce(sc, dirs, 6, tr, nb)
    _check_norm(T, Tref, allow.max(axis=1), 1e-3 * oracle.unoccluded_norm(6))


# ---- backward of the bounces (Eq. 33-35, index matrix fixed) -------------------------------
@pytest.mark.parametrize("order,nb", [(3, 1), (2, 3), (6, 2)])
def test_bounce_backward_matches_autograd(order, nb):
    """dT -> dP, d_albedo, d_normals through the bounces against FP64 autograd of the
    bounce restatement on the GPU's own P and index matrix."""
    from oracle import transfer_torch as TT

    sc = _crowded(1200, 40 + order)
    dirs = S.direction_set(64, 6)
    g = _gt(sc)
    st = api.Status()
    bvh = api.build_bvh(g, status=st)
    d = torch.from_numpy(dirs).cuda()
    out = api.precompute_transfer(g, bvh, d, order, bounce=True, n_bounces=nb, status=st)
    C = (order + 1) ** 2
    dT = np.random.default_rng(order + nb).standard_normal((sc.n, 3, C)).astype(np.float32)
    dP, da, dn = api.bounce_backward(g, d, order, out["P"], out["idx"], torch.from_numpy(dT).cuda(), nb, status=st)
    torch.cuda.synchronize()
    assert st.read() == 0
    idx = out["idx"].cpu().numpy()
    assert (idx >= 0).mean() > 0.1
    t = lambda a, rg=False: torch.tensor(np.asarray(a, np.float64), requires_grad=rg)
    P, rho, nrm = t(out["P"].cpu().numpy(), True), t(sc.albedo, True), t(sc.normals, True)
    T = TT.bounce_T(P, idx, dirs, nrm, rho, nb)
    np.testing.assert_allclose(out["T"].cpu().numpy(), T.detach().numpy(), rtol=0,
                               atol=2e-6 * float(T.detach().abs().max()))
    ref = torch.autograd.grad((T * torch.as_tensor(dT.astype(np.float64))).sum(), (P, rho, nrm))
    for got, r, name in zip((dP, da, dn), ref, ("dP", "d_albedo", "d_normals")):
        got = got.cpu().numpy().astype(np.float64)
        r = r.numpy()
        assert np.linalg.norm(got - r) <= 1e-5 * np.linalg.norm(r), (name, np.linalg.norm(got - r) / np.linalg.norm(r))
        assert np.linalg.norm(r) > 0


def test_bounce_transfer_gradient_to_the_gaussians():
    """L = sum(W * T) for the one-bounce T: the geometry, normal and albedo gradients of
    BounceTransfer (bounce backward, then the transfer backward) against FP64 autograd of the
    brute-force P chained into the bounce restatement, with the GPU's index matrix held fixed."""
    from oracle import transfer_torch as TT

    sc = _crowded(260, 17)
    dirs = S.direction_set(40, 5)
    order = 2
    C = (order + 1) ** 2
    fields = ("means", "scales", "quats", "opacity", "normals", "albedo")
    gp = [torch.tensor(np.asarray(getattr(sc, f), np.float32), device="cuda", requires_grad=True) for f in fields]
    d = torch.from_numpy(dirs).cuda()
    T = api.bounce_transfer(*gp, d, order, 1, 0.0)
    W = np.random.default_rng(3).standard_normal((sc.n, 3, C))
    (T * torch.as_tensor(W, dtype=torch.float32, device="cuda")).sum().backward()
    gpu = {f: p.grad.cpu().numpy().astype(np.float64) for f, p in zip(fields, gp)}
    # the index matrix of the same forward, held fixed in the reference
    g = _gt(sc)
    idx = api.precompute_transfer(g, api.build_bvh(g), d, order, bounce=True, t_min=0.0)["idx"].cpu().numpy()
    ps = [torch.tensor(np.asarray(getattr(sc, f), np.float64), requires_grad=True) for f in fields]
    P = TT.transfer_P(*ps[:5], dirs, oracle.sh(order, dirs))
    Tr = TT.bounce_T(P, idx, dirs, ps[4], ps[5], 1)
    np.testing.assert_allclose(T.detach().cpu().numpy(), Tr.detach().numpy(), rtol=0, atol=1e-4)
    ref = torch.autograd.grad((Tr * torch.as_tensor(W)).sum(), ps)
    top = max(np.linalg.norm(r.numpy()) for r in ref)
    for f, r in zip(fields, ref):
        r = r.numpy()
        nb = max(np.linalg.norm(r), 1e-3 * top)
        assert np.linalg.norm(gpu[f] - r) <= 2e-3 * nb, (f, np.linalg.norm(gpu[f] - r) / nb)
    assert np.linalg.norm(ref[5].numpy()) > 0 and np.linalg.norm(ref[3].numpy()) > 0


# ---- backward of the glossy matrices (Eq. 40) ----------------------------------------------
@pytest.mark.parametrize("order", [3, 5])
def test_glossy_backward_matches_autograd(order):
    """dM -> dV, d_roughness, d_metallic, d_normals against FP64 autograd of the glossy matrices on
    the GPU's own visibility; non-glossy rows stay zero."""
    from oracle import transfer_torch as TT

    sc = S.surface_scene(900, 80 + order)
    rng = np.random.default_rng(order)
    sc.glossy_mask = (rng.random(sc.n) < 0.2).astype(np.uint8)
    sc.roughness = rng.uniform(0.25, 0.9, sc.n).astype(np.float32)
    sc.metallic = rng.uniform(0.0, 1.0, sc.n).astype(np.float32)
    dirs = S.direction_set(48, 9)
    g = _gt(sc)
    st = api.Status()
    bvh = api.build_bvh(g, status=st)
    d = torch.from_numpy(dirs).cuda()
    V = api.precompute_visibility(g, bvh, d, order, status=st)["V"]
    gids = np.nonzero(sc.glossy_mask)[0]
    C = (order + 1) ** 2
    dM = rng.standard_normal((gids.size, C, C)).astype(np.float32)
    dV, dr, dm, dn = api.glossy_backward(g, d, order, V, torch.from_numpy(dM).cuda(), status=st)
    torch.cuda.synchronize()
    assert st.read() == 0
    t = lambda a: torch.tensor(np.asarray(a, np.float64), requires_grad=True)
    Vg, ng, rg, mg = (t(V.cpu().numpy()[gids]), t(sc.normals[gids]), t(sc.roughness[gids]), t(sc.metallic[gids]))
    M = TT.glossy_M(Vg, ng, rg, mg, dirs, oracle.sh(order, dirs))
    ref = torch.autograd.grad((M * torch.as_tensor(dM.astype(np.float64))).sum(), (Vg, ng, rg, mg))
    got = [x.cpu().numpy().astype(np.float64) for x in (dV, dn, dr, dm)]
    other = np.ones(sc.n, bool)
    other[gids] = False
    for name, a, r, tol in zip(("dV", "d_normals", "d_roughness", "d_metallic"), got, ref, (2e-4, 2e-3, 5e-4, 2e-4)):
        r = r.numpy()
        assert np.all(a[other] == 0), name
        a = a[gids]
        assert np.linalg.norm(a - r) <= tol * np.linalg.norm(r), (name, np.linalg.norm(a - r) / np.linalg.norm(r))
        assert np.linalg.norm(r) > 0, name


def test_glossy_transfer_gradient_to_the_gaussians():
    """L = sum(Wp * P) + sum(Wm * M): the geometry, normal, roughness and metallic gradients of
    GlossyTransfer (glossy backward, then the transfer backward with its visibility gradient)
    against FP64 autograd of the brute-force visibility chained into P and the glossy matrices."""
    from oracle import transfer_torch as TT

    sc = _crowded(220, 19)
    rng = np.random.default_rng(19)
    sc.glossy_mask = (rng.random(sc.n) < 0.3).astype(np.uint8)
    sc.roughness = rng.uniform(0.3, 0.9, sc.n).astype(np.float32)
    sc.metallic = rng.uniform(0.0, 1.0, sc.n).astype(np.float32)
    dirs = S.direction_set(32, 5)
    order = 2
    C = (order + 1) ** 2
    fields = ("means", "scales", "quats", "opacity", "normals", "roughness", "metallic")
    gp = [torch.tensor(np.asarray(getattr(sc, f), np.float32), device="cuda", requires_grad=True) for f in fields]
    mask = torch.from_numpy(sc.glossy_mask).cuda()
    alb = torch.from_numpy(np.asarray(sc.albedo, np.float32)).cuda()
    d = torch.from_numpy(dirs).cuda()
    P, M = api.glossy_transfer(*gp, mask, alb, d, order, 0.0)
    gids = np.nonzero(sc.glossy_mask)[0]
    Wp = rng.standard_normal((sc.n, C))
    Wm = rng.standard_normal((gids.size, C, C))
    loss = (P * torch.as_tensor(Wp, dtype=torch.float32, device="cuda")).sum() + \
        (M * torch.as_tensor(Wm, dtype=torch.float32, device="cuda")).sum()
    loss.backward()
    gpu = {f: p.grad.cpu().numpy().astype(np.float64) for f, p in zip(fields, gp)}
    ps = [torch.tensor(np.asarray(getattr(sc, f), np.float64), requires_grad=True) for f in fields]
    Y = oracle.sh(order, dirs)
    V = TT.transfer_V(*ps[:5], dirs)
    dd = torch.as_tensor(np.asarray(dirs, np.float64))
    c = ps[4] @ dd.T
    Pr = torch.where((c > 0).detach(), 4.0 * math.pi / len(dirs) * V * c, torch.zeros_like(c)) @ torch.as_tensor(Y)
    gi = torch.as_tensor(gids)
    Mr = TT.glossy_M(V[gi], ps[4][gi], ps[5][gi], ps[6][gi], dirs, Y)
    np.testing.assert_allclose(M.detach().cpu().numpy(), Mr.detach().numpy(), rtol=0,
                               atol=1e-4 * float(Mr.detach().abs().max()))
    ref = torch.autograd.grad((Pr * torch.as_tensor(Wp)).sum() + (Mr * torch.as_tensor(Wm)).sum(), ps)
    top = max(np.linalg.norm(r.numpy()) for r in ref)
    for f, r in zip(fields, ref):
        r = r.numpy()
        nb = max(np.linalg.norm(r), 1e-3 * top)
        assert np.linalg.norm(gpu[f] - r) <= 2e-3 * nb, (f, np.linalg.norm(gpu[f] - r) / nb)
    assert all(np.linalg.norm(ref[k].numpy()) > 0 for k in (0, 3, 4, 5, 6))
