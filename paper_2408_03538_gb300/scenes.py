"""Seeded synthetic inputs: Gaussian scenes, the shared direction set, lights and cameras.

This module only draws inputs. It holds none of the method's arithmetic (no SH, no
transmittance, no projection), so both the CUDA path and the FP64 oracle may take their
inputs from it. Every array it returns is a plain numpy array (FP32 unless noted).

The paper trains its Gaussians on TensoIR-Synthetic, DTU and Mip-NeRF 360 (Sec. 5.1);
none of that data is available here, so these generators stand in for it with the
shapes, scale distributions and surface structure of those scenes:

* ``isotropic_scene``: centres uniform in [-1,1]^3, isotropic scales lognormal(-3, 0.3),
  opacity U[0.2,0.9], unit normals uniform on the sphere, albedo U[0,1]^3.
* ``surface_scene``: Gaussians sampled area-proportionally on a unit sphere standing on a
  ground plane z=0 over [-4,4]^2 with three boxes, flattened along the surface normal
  (axis ratio 1:1 to 10:1) and rotated so their local z axis is the surface normal.
* ``tiled_scene``: the surface scene repeated 10 times on a 5x2 grid (spacing 12) with a
  uniformly random rotation per instance, 30 % of the splats glossy.
* ``batched_scenes``: 32 isotropic scenes with Gaussian counts log-uniform in [1e4, 5e5].
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 2408035380


def rng_for(seed: int) -> np.random.Generator:
    """PCG64 stream for ``seed`` (stable across numpy versions and platforms)."""
    return np.random.Generator(np.random.PCG64(int(seed)))


def config_seed(config_index: int) -> int:
    return SEED_BASE + int(config_index)


@dataclass
class Scene:
    """Structure-of-arrays Gaussian set (FP32, C-contiguous).

    means[N,3], scales[N,3] (linear standard deviations along the local axes),
    quats[N,4] as (w,x,y,z), opacity[N], normals[N,3] (unit), albedo[N,3],
    roughness[N], metallic[N], glossy_mask[N] (uint8).
    """

    means: np.ndarray
    scales: np.ndarray
    quats: np.ndarray
    opacity: np.ndarray
    normals: np.ndarray
    albedo: np.ndarray
    roughness: np.ndarray
    metallic: np.ndarray
    glossy_mask: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def subset(self, idx) -> "Scene":
        idx = np.asarray(idx)
        return Scene(*(np.ascontiguousarray(getattr(self, f)[idx]) for f in FIELDS), meta=dict(self.meta))

    def arrays(self) -> dict:
        return {f: getattr(self, f) for f in FIELDS}


FIELDS = ("means", "scales", "quats", "opacity", "normals", "albedo", "roughness", "metallic", "glossy_mask")


def _finish(means, scales, quats, opacity, normals, albedo, roughness=None, metallic=None, glossy=None, meta=None):
    n = means.shape[0]
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return Scene(
        means=f32(means),
        scales=f32(scales),
        quats=f32(quats),
        opacity=f32(opacity),
        normals=f32(normals),
        albedo=f32(albedo),
        roughness=f32(roughness if roughness is not None else np.full(n, 0.5)),
        metallic=f32(metallic if metallic is not None else np.zeros(n)),
        glossy_mask=np.ascontiguousarray(glossy if glossy is not None else np.zeros(n), dtype=np.uint8),
        meta=meta or {},
    )


def unit_vectors(rng: np.random.Generator, n: int) -> np.ndarray:
    v = rng.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v


def random_quats(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform random rotations (Shoemake 1992, 'Uniform random rotations'), (w,x,y,z), w >= 0."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    a, b = np.sqrt(1 - u1), np.sqrt(u1)
    q = np.stack([a * np.sin(2 * np.pi * u2), a * np.cos(2 * np.pi * u2),
                  b * np.sin(2 * np.pi * u3), b * np.cos(2 * np.pi * u3)], axis=1)  # (x,y,z,w)
    q = np.concatenate([q[:, 3:4], q[:, :3]], axis=1)
    q[q[:, 0] < 0] *= -1
    return q


def _frame_to_quat(m: np.ndarray) -> np.ndarray:
    """(w,x,y,z) unit quaternions of proper rotation matrices m[N,3,3] (columns = local axes)."""
    n = m.shape[0]
    q = np.zeros((n, 4))
    tr = m[:, 0, 0] + m[:, 1, 1] + m[:, 2, 2]
    # pick the numerically largest of w,x,y,z per matrix
    cand = np.stack([tr, m[:, 0, 0], m[:, 1, 1], m[:, 2, 2]], axis=1)
    k = np.argmax(cand, axis=1)
    for case in range(4):
        s_ = k == case
        if not np.any(s_):
            continue
        a = m[s_]
        if case == 0:
            r = np.sqrt(1.0 + a[:, 0, 0] + a[:, 1, 1] + a[:, 2, 2]) * 2
            q[s_] = np.stack([0.25 * r, (a[:, 2, 1] - a[:, 1, 2]) / r, (a[:, 0, 2] - a[:, 2, 0]) / r,
                              (a[:, 1, 0] - a[:, 0, 1]) / r], axis=1)
        elif case == 1:
            r = np.sqrt(1.0 + a[:, 0, 0] - a[:, 1, 1] - a[:, 2, 2]) * 2
            q[s_] = np.stack([(a[:, 2, 1] - a[:, 1, 2]) / r, 0.25 * r, (a[:, 0, 1] + a[:, 1, 0]) / r,
                              (a[:, 0, 2] + a[:, 2, 0]) / r], axis=1)
        elif case == 2:
            r = np.sqrt(1.0 + a[:, 1, 1] - a[:, 0, 0] - a[:, 2, 2]) * 2
            q[s_] = np.stack([(a[:, 0, 2] - a[:, 2, 0]) / r, (a[:, 0, 1] + a[:, 1, 0]) / r, 0.25 * r,
                              (a[:, 1, 2] + a[:, 2, 1]) / r], axis=1)
        else:
            r = np.sqrt(1.0 + a[:, 2, 2] - a[:, 0, 0] - a[:, 1, 1]) * 2
            q[s_] = np.stack([(a[:, 1, 0] - a[:, 0, 1]) / r, (a[:, 0, 2] + a[:, 2, 0]) / r,
                              (a[:, 1, 2] + a[:, 2, 1]) / r, 0.25 * r], axis=1)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    q[q[:, 0] < 0] *= -1
    return q


def isotropic_scene(n: int, seed: int) -> Scene:
    """Plain-method scene: uniform centres in [-1,1]^3, isotropic lognormal(-3,0.3) scales."""
    rng = rng_for(seed)
    means = rng.uniform(-1.0, 1.0, (n, 3))
    s = np.exp(rng.normal(-3.0, 0.3, n))
    scales = np.repeat(s[:, None], 3, axis=1)
    quats = random_quats(rng, n)
    opacity = rng.uniform(0.2, 0.9, n)
    normals = unit_vectors(rng, n)
    albedo = rng.uniform(0.0, 1.0, (n, 3))
    return _finish(means, scales, quats, opacity, normals, albedo,
                   meta={"generator": "isotropic", "n": n, "seed": seed})


def _boxes(rng):
    boxes = []
    while len(boxes) < 3:
        size = rng.uniform(0.4, 1.0, 3)
        yaw = rng.uniform(0.0, 2 * np.pi)
        c = rng.uniform(-3.0, 3.0, 2)
        if np.linalg.norm(c) < 1.0 + 0.75:
            continue
        if any(np.linalg.norm(c - b[0]) < 1.5 for b in boxes):
            continue
        boxes.append((c, size, yaw))
    return boxes


def _in_footprint(xy, boxes):
    inside = np.zeros(xy.shape[0], dtype=bool)
    for c, size, yaw in boxes:
        d = xy - c
        cs, sn = np.cos(yaw), np.sin(yaw)
        lx = cs * d[:, 0] + sn * d[:, 1]
        ly = -sn * d[:, 0] + cs * d[:, 1]
        inside |= (np.abs(lx) <= size[0] / 2) & (np.abs(ly) <= size[1] / 2)
    return inside


def surface_points(rng: np.random.Generator, n: int):
    """Area-proportional points and outward normals on sphere + ground plane + 3 boxes."""
    boxes = _boxes(rng)
    # surfaces: 0 ground, 1 sphere, then per box 5 faces (top, +x, -x, +y, -y in box frame)
    areas = [64.0 - sum(b[1][0] * b[1][1] for b in boxes), 4 * np.pi]
    for c, size, yaw in boxes:
        sx, sy, sz = size
        areas += [sx * sy, sy * sz, sy * sz, sx * sz, sx * sz]
    areas = np.asarray(areas)
    which = rng.choice(len(areas), size=n, p=areas / areas.sum())
    pts = np.zeros((n, 3))
    nrm = np.zeros((n, 3))
    # ground (rejection outside box footprints)
    g = np.nonzero(which == 0)[0]
    fill = np.zeros((0, 2))
    while fill.shape[0] < g.size:
        cand = rng.uniform(-4.0, 4.0, (2 * (g.size - fill.shape[0]) + 16, 2))
        cand = cand[~_in_footprint(cand, boxes)]
        fill = np.concatenate([fill, cand], axis=0)
    pts[g, :2] = fill[: g.size]
    nrm[g] = (0.0, 0.0, 1.0)
    # sphere
    sp = np.nonzero(which == 1)[0]
    u = unit_vectors(rng, sp.size)
    pts[sp] = u + np.array([0.0, 0.0, 1.0])
    nrm[sp] = u
    # boxes
    for bi, (c, size, yaw) in enumerate(boxes):
        sx, sy, sz = size
        cs, sn = np.cos(yaw), np.sin(yaw)
        rot = np.array([[cs, -sn, 0.0], [sn, cs, 0.0], [0.0, 0.0, 1.0]])
        for f in range(5):
            ids = np.nonzero(which == 2 + 5 * bi + f)[0]
            if ids.size == 0:
                continue
            a, b = rng.random(ids.size) - 0.5, rng.random(ids.size) - 0.5
            loc = np.zeros((ids.size, 3))
            ln = np.zeros(3)
            if f == 0:
                loc[:, 0], loc[:, 1], loc[:, 2] = a * sx, b * sy, sz
                ln[2] = 1
            elif f in (1, 2):
                sgn = 1.0 if f == 1 else -1.0
                loc[:, 0], loc[:, 1], loc[:, 2] = sgn * sx / 2, a * sy, (b + 0.5) * sz
                ln[0] = sgn
            else:
                sgn = 1.0 if f == 3 else -1.0
                loc[:, 0], loc[:, 1], loc[:, 2] = a * sx, sgn * sy / 2, (b + 0.5) * sz
                ln[1] = sgn
            pts[ids] = loc @ rot.T + np.array([c[0], c[1], 0.0])
            nrm[ids] = rot @ ln
    return pts, nrm, boxes


def surface_scene(n: int, seed: int) -> Scene:
    """Anisotropic Gaussians on a synthetic surface (sphere over a ground plane with 3 boxes)."""
    rng = rng_for(seed)
    pts, nrm, boxes = surface_points(rng, n)
    # orthonormal tangent frame with a random spin about the normal
    helper = np.where(np.abs(nrm[:, 2:3]) < 0.9, np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]]))
    t1 = np.cross(helper, nrm)
    t1 /= np.linalg.norm(t1, axis=1, keepdims=True)
    t2 = np.cross(nrm, t1)
    spin = rng.uniform(0.0, 2 * np.pi, n)[:, None]
    a1 = np.cos(spin) * t1 + np.sin(spin) * t2
    a2 = np.cross(nrm, a1)
    frame = np.stack([a1, a2, nrm], axis=2)  # columns: local x, y, z(=normal)
    quats = _frame_to_quat(frame)
    st = np.exp(rng.normal(-3.0, 0.3, (n, 2)))
    sn = st.min(axis=1) / rng.uniform(1.0, 10.0, n)
    scales = np.concatenate([st, sn[:, None]], axis=1)
    opacity = rng.uniform(0.2, 0.9, n)
    albedo = rng.uniform(0.0, 1.0, (n, 3))
    return _finish(pts, scales, quats, opacity, nrm, albedo,
                   meta={"generator": "surface", "n": n, "seed": seed,
                         "boxes": [(b[0].tolist(), b[1].tolist(), float(b[2])) for b in boxes]})


def _quat_mul(a, b):
    w1, x1, y1, z1 = a[..., 0], a[..., 1], a[..., 2], a[..., 3]
    w2, x2, y2, z2 = b[..., 0], b[..., 1], b[..., 2], b[..., 3]
    return np.stack([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                     w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                     w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2], axis=-1)


def random_rotation_matrices(rng: np.random.Generator, n: int) -> np.ndarray:
    """Haar-uniform proper rotations [n,3,3] from the QR factorisation of Gaussian matrices."""
    a = rng.standard_normal((n, 3, 3))
    q, r = np.linalg.qr(a)
    q = q * np.sign(np.diagonal(r, axis1=1, axis2=2))[:, None, :]
    det = np.linalg.det(q)
    q[det < 0, :, 0] *= -1
    return q


def tiled_scene(seed: int, base_n: int = 100_000, copies=(5, 2), spacing: float = 12.0,
                glossy_fraction: float = 0.3) -> Scene:
    """The surface scene repeated on a grid, one uniform random rotation per instance."""
    base = surface_scene(base_n, seed)
    rng = rng_for(seed + 7919)
    inst_m = random_rotation_matrices(rng, copies[0] * copies[1])
    inst_q = _frame_to_quat(inst_m)
    parts = {f: [] for f in FIELDS}
    k = 0
    for gx in range(copies[0]):
        for gy in range(copies[1]):
            q, m = inst_q[k], inst_m[k]
            k += 1
            off = np.array([(gx - (copies[0] - 1) / 2) * spacing, (gy - (copies[1] - 1) / 2) * spacing, 0.0])
            parts["means"].append(base.means.astype(np.float64) @ m.T + off)
            parts["normals"].append(base.normals.astype(np.float64) @ m.T)
            parts["quats"].append(_quat_mul(np.broadcast_to(q, base.quats.shape), base.quats.astype(np.float64)))
            for f in ("scales", "opacity", "albedo"):
                parts[f].append(getattr(base, f))
    cat = {f: np.concatenate(v, axis=0) for f, v in parts.items() if v}
    n = cat["means"].shape[0]
    qq = cat["quats"]
    qq[qq[:, 0] < 0] *= -1
    nrm = cat["normals"] / np.linalg.norm(cat["normals"], axis=1, keepdims=True)
    glossy = (rng.random(n) < glossy_fraction).astype(np.uint8)
    rough = rng.uniform(0.1, 0.6, n)
    metal = rng.uniform(0.0, 1.0, n)
    return _finish(cat["means"], cat["scales"], qq, cat["opacity"], nrm, cat["albedo"], rough, metal, glossy,
                   meta={"generator": "tiled", "n": n, "seed": seed})


def batched_sizes(seed: int, n_scenes: int = 32, lo: float = 1e4, hi: float = 5e5) -> list:
    rng = rng_for(seed)
    return [int(round(math.exp(v))) for v in rng.uniform(math.log(lo), math.log(hi), n_scenes)]


def batched_scenes(seed: int, n_scenes: int = 32, lo: float = 1e4, hi: float = 5e5) -> list:
    sizes = batched_sizes(seed, n_scenes, lo, hi)
    return [isotropic_scene(nb, seed * 1000 + b + 1) for b, nb in enumerate(sizes)]


def concat_scenes(scenes) -> tuple:
    """Concatenate scenes into one SoA set plus int64 offsets [B+1]."""
    offs = np.zeros(len(scenes) + 1, dtype=np.int64)
    offs[1:] = np.cumsum([s.n for s in scenes])
    merged = Scene(*(np.ascontiguousarray(np.concatenate([getattr(s, f) for s in scenes], axis=0)) for f in FIELDS),
                   meta={"generator": "batched", "sizes": [s.n for s in scenes]})
    return merged, offs


def direction_set(n_dirs: int, seed: int) -> np.ndarray:
    """The shared set of S sphere directions [S,3] (FP32), one per equal-area band.

    Direction k lies in the band z in (1-2(k+1)/S, 1-2k/S] at a jittered height, with its
    azimuth advanced by the golden-ratio fraction (a jittered spherical Fibonacci set).
    The jitter is drawn from the PCG64 stream of ``seed``. Computed in FP64 and rounded once.
    """
    rng = rng_for(seed)
    u = rng.random(n_dirs)
    v = rng.random(n_dirs)
    k = np.arange(n_dirs, dtype=np.float64)
    z = 1.0 - 2.0 * (k + u) / n_dirs
    golden = (math.sqrt(5.0) - 1.0) / 2.0
    phi = 2.0 * math.pi * np.mod(k * golden + v / n_dirs, 1.0)
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    d = np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)
    return np.ascontiguousarray(d.astype(np.float32))


def sh_count(order: int) -> int:
    return (order + 1) * (order + 1)


def env_lights(k: int, order: int, seed: int) -> np.ndarray:
    """k random RGB environment lights in real SH, [k,3,C] FP32.

    The DC coefficient is U[0.5,1.5] per channel; band l>0 coefficients are N(0,(0.3/(l+1))^2).
    """
    rng = rng_for(seed)
    c = sh_count(order)
    out = np.zeros((k, 3, c))
    out[:, :, 0] = rng.uniform(0.5, 1.5, (k, 3))
    for l in range(1, order + 1):
        for m in range(-l, l + 1):
            out[:, :, l * l + l + m] = rng.normal(0.0, 0.3 / (l + 1), (k, 3))
    return np.ascontiguousarray(out.astype(np.float32))


@dataclass
class Camera:
    """Pinhole camera. ``rot``/``trans`` map world to camera: x_c = rot @ x_w + trans.

    Camera axes: x right, y down, z forward. Pixel (px,py) has its centre at
    (fx*x/z + cx, fy*y/z + cy) == (px, py).
    """

    rot: np.ndarray
    trans: np.ndarray
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    near: float = 0.2
    position: np.ndarray = None


def look_at_camera(eye, target, fov_y_deg: float, width: int, height: int, up=(0.0, 0.0, 1.0),
                   near: float = 0.2) -> Camera:
    eye = np.asarray(eye, dtype=np.float64)
    target = np.asarray(target, dtype=np.float64)
    f = target - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, dtype=np.float64))
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    rot = np.stack([r, d, f], axis=0)
    trans = -rot @ eye
    fy = 0.5 * height / math.tan(math.radians(fov_y_deg) / 2)
    fx = fy
    return Camera(rot=rot.astype(np.float32), trans=trans.astype(np.float32), fx=float(np.float32(fx)),
                  fy=float(np.float32(fy)), cx=(width - 1) / 2.0, cy=(height - 1) / 2.0, width=width,
                  height=height, near=near, position=eye.astype(np.float32))


# Workload recipes --------------------------------------------------------------------------------

WORKLOADS = {
    "tiny-1k": dict(config=0, generator="isotropic", n=1024, order=2, n_dirs=64, bounce=False, lights=1,
                    width=256, height=256, eye=(0.0, -3.5, 1.5), target=(0.0, 0.0, 0.0), fov=50.0),
    "surface-100k": dict(config=1, generator="surface", n=100_000, order=3, n_dirs=256, bounce=True, lights=1,
                         width=1920, height=1080, eye=(0.0, -7.0, 3.0), target=(0.0, 0.0, 0.8), fov=45.0),
    "tiled-1m-glossy": dict(config=2, generator="tiled", n=1_000_000, order=3, n_dirs=256, bounce=True, lights=64,
                            width=1920, height=1080, eye=(0.0, -40.0, 14.0), target=(0.0, 0.0, 0.0), fov=45.0),
    "diff-300k": dict(config=3, generator="isotropic", n=300_000, order=3, n_dirs=128, bounce=False, lights=1,
                      width=1920, height=1080, eye=(0.0, -3.5, 1.5), target=(0.0, 0.0, 0.0), fov=50.0),
    "batched-32": dict(config=4, generator="batched", n=None, order=3, n_dirs=128, bounce=False, lights=8,
                       width=1280, height=720, eye=(0.0, -3.5, 1.5), target=(0.0, 0.0, 0.0), fov=50.0),
}


def make_scene(name: str, n: int | None = None) -> Scene:
    w = WORKLOADS[name]
    seed = config_seed(w["config"])
    n = n if n is not None else w["n"]
    if w["generator"] == "isotropic":
        return isotropic_scene(n, seed)
    if w["generator"] == "surface":
        return surface_scene(n, seed)
    if w["generator"] == "tiled":
        return tiled_scene(seed)
    raise ValueError(name)


def make_camera(name: str, width: int | None = None, height: int | None = None) -> Camera:
    w = WORKLOADS[name]
    return look_at_camera(w["eye"], w["target"], w["fov"], width or w["width"], height or w["height"])
