"""PyTorch-facing wrappers of libprtgs (argument marshalling only).

PyTorch supplies device memory (outputs and workspaces via the caching allocator) and the
current CUDA stream; every step of the computation runs in the library's own kernels.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib as L

DEFAULT_T_MIN = 2.0 ** -30


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "tensors passed to libprtgs must be contiguous CUDA tensors"
    return ctypes.c_void_p(t.data_ptr())


def _ws(nbytes: int, device):
    if nbytes == 0:
        return None, 0
    t = torch.empty(int(nbytes), dtype=torch.uint8, device=device)
    return t, int(nbytes)


def sh_count(order: int) -> int:
    return (order + 1) ** 2


@dataclass
class GaussianTensors:
    """Device SoA Gaussian set (FP32; glossy_mask uint8)."""

    means: torch.Tensor
    scales: torch.Tensor
    quats: torch.Tensor
    opacity: torch.Tensor
    normals: torch.Tensor
    albedo: torch.Tensor
    roughness: torch.Tensor = None
    metallic: torch.Tensor = None
    glossy_mask: torch.Tensor = None

    @property
    def n(self):
        return int(self.means.shape[0])

    def struct(self) -> L.Gaussians:
        return L.Gaussians(self.n, _ptr(self.means), _ptr(self.scales), _ptr(self.quats), _ptr(self.opacity),
                           _ptr(self.normals), _ptr(self.albedo), _ptr(self.roughness), _ptr(self.metallic),
                           _ptr(self.glossy_mask))

    @staticmethod
    def from_scene(scene, device="cuda"):
        f = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
        return GaussianTensors(f(scene.means), f(scene.scales), f(scene.quats), f(scene.opacity), f(scene.normals),
                               f(scene.albedo), f(scene.roughness), f(scene.metallic), f(scene.glossy_mask))

    def with_(self, **kw):
        d = dict(self.__dict__)
        d.update(kw)
        return GaussianTensors(**d)


class Status:
    """A device int32 status word (PRTGS_STATUS_* bits)."""

    def __init__(self, device="cuda"):
        self.t = torch.zeros(1, dtype=torch.int32, device=device)

    def ptr(self):
        return _ptr(self.t)

    def read(self) -> int:
        rc = L.load().prtgs_read_status(self.ptr(), _stream())
        if rc < 0:
            L.check(rc, "prtgs_read_status")
        return rc


# ------------------------------------------------------------------------------------------
# BVH
# ------------------------------------------------------------------------------------------
class Bvh:
    def __init__(self, n: int, scene_offsets: torch.Tensor):
        lib = L.load()
        self.n = n
        self.offsets = scene_offsets.to(dtype=torch.int64).contiguous()
        self.n_scenes = int(self.offsets.numel() - 1)
        nbytes = lib.prtgs_bvh_bytes(n, self.n_scenes)
        self.buffer = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=self.offsets.device)
        self.s = L.BVH()
        L.check(lib.prtgs_bvh_init(_ptr(self.buffer), nbytes, n, self.n_scenes, _ptr(self.offsets),
                                   ctypes.byref(self.s)), "prtgs_bvh_init")

    def view(self, field, dtype, shape):
        """Tensor view of one BVH array (for tests)."""
        lib_ptr = getattr(self.s, field)
        off = lib_ptr - self.buffer.data_ptr()
        count = int(np.prod(shape))
        nbytes = count * torch.empty(0, dtype=dtype).element_size()
        return self.buffer[off:off + nbytes].view(dtype).view(*shape)


def build_bvh(g: GaussianTensors, scene_offsets: torch.Tensor | None = None, status: Status | None = None) -> Bvh:
    lib = L.load()
    if scene_offsets is None:
        scene_offsets = torch.tensor([0, g.n], dtype=torch.int64, device=g.means.device)
    bvh = Bvh(g.n, scene_offsets)
    ws, nb = _ws(lib.prtgs_build_bvh_workspace_size(g.n, bvh.n_scenes), g.means.device)
    gs = g.struct()
    L.check(lib.prtgs_build_bvh(ctypes.byref(gs), ctypes.byref(bvh.s), status.ptr() if status else None, _ptr(ws), nb,
                                _stream()), "prtgs_build_bvh")
    bvh._ws = ws  # keep alive until the stream has consumed it
    return bvh


# ------------------------------------------------------------------------------------------
# Transfer
# ------------------------------------------------------------------------------------------
def precompute_transfer(g: GaussianTensors, bvh: Bvh, dirs: torch.Tensor, order: int, shadow: bool = True,
                        bounce: bool = False, glossy: bool = False, t_min: float = DEFAULT_T_MIN,
                        same_surface_t: float = 1.0, status: Status | None = None, out: dict | None = None,
                        stats: torch.Tensor | None = None, index_buffer: int = 0, n_bounces: int = 1,
                        walk: int = 0, packet_dirs: int = 0):
    """Transfer vectors P [n,C], and with ``bounce`` T [n,3,C] (``n_bounces`` self-transfer
    bounces over the index matrix) and idx [n,S]; with ``glossy`` the C x C matrices
    M [n_glossy,C,C] of the glossy splats (in increasing index order). ``walk``: 0 = warp
    packets of parallel rays (default), 1 = one ray per lane; the results are the same."""
    lib = L.load()
    dev = g.means.device
    S = int(dirs.shape[0])
    C = sh_count(order)
    flags = (L.SHADOW if shadow else 0) | (L.BOUNCE if bounce else 0) | (L.GLOSSY if glossy else 0)
    n_glossy = int(g.glossy_mask.sum().item()) if glossy else 0
    out = out or {}
    P = out.get("P") if out.get("P") is not None else torch.empty((g.n, C), dtype=torch.float32, device=dev)
    T = idx = M = None
    if bounce:
        T = out.get("T") if out.get("T") is not None else torch.empty((g.n, 3, C), dtype=torch.float32, device=dev)
        idx = out.get("idx") if out.get("idx") is not None else torch.empty((g.n, S), dtype=torch.int32, device=dev)
    if glossy:
        M = torch.empty((max(n_glossy, 1), C, C), dtype=torch.float32, device=dev)
    p = L.TransferParams(order, S, _ptr(dirs), float(t_min), float(same_surface_t), flags, int(index_buffer),
                         _ptr(stats), int(n_bounces), int(walk), int(packet_dirs))
    ws, nb = _ws(lib.prtgs_transfer_workspace_size(g.n, n_glossy, ctypes.byref(p)), dev)
    gs = g.struct()
    L.check(lib.prtgs_precompute_transfer(ctypes.byref(gs), ctypes.byref(bvh.s), ctypes.byref(p), _ptr(P), _ptr(T),
                                          _ptr(idx), _ptr(M), n_glossy, status.ptr() if status else None, _ptr(ws),
                                          nb, _stream()), "prtgs_precompute_transfer")
    res = {"P": P, "_ws": ws}
    if bounce:
        res.update(T=T, idx=idx)
    if glossy:
        res.update(M=M[:n_glossy], n_glossy=n_glossy)
    return res


def precompute_transfer_backward(g: GaussianTensors, bvh: Bvh, dirs: torch.Tensor, order: int, dP: torch.Tensor,
                                 shadow: bool = True, t_min: float = DEFAULT_T_MIN, status: Status | None = None,
                                 stats: torch.Tensor | None = None, dV: torch.Tensor | None = None):
    """Gradients of a loss through P [n,C] (shadowed diffuse transfer) and, optionally, through the
    rays' visibility directly (dV [n,S], e.g. from the glossy matrices) to the Gaussians: dict of
    d_means [n,3], d_scales [n,3], d_quats [n,4], d_opacity [n], d_normals [n,3]."""
    lib = L.load()
    dev = g.means.device
    n = g.n
    f32 = dict(dtype=torch.float32, device=dev)
    grads = {"d_means": torch.empty((n, 3), **f32), "d_scales": torch.empty((n, 3), **f32),
             "d_quats": torch.empty((n, 4), **f32), "d_opacity": torch.empty((n,), **f32),
             "d_normals": torch.empty((n, 3), **f32)}
    dP = dP.contiguous() if dP is not None else None
    p = L.TransferParams(order, int(dirs.shape[0]), _ptr(dirs), float(t_min), 1.0, L.SHADOW if shadow else 0, 0,
                         _ptr(stats))
    ws, nb = _ws(lib.prtgs_transfer_backward_workspace_size(n, ctypes.byref(p)), dev)
    gs = g.struct()
    if dV is None:
        L.check(lib.prtgs_precompute_transfer_backward(
            ctypes.byref(gs), ctypes.byref(bvh.s), ctypes.byref(p), _ptr(dP), _ptr(grads["d_means"]),
            _ptr(grads["d_scales"]), _ptr(grads["d_quats"]), _ptr(grads["d_opacity"]), _ptr(grads["d_normals"]),
            status.ptr() if status else None, _ptr(ws), nb, _stream()), "prtgs_precompute_transfer_backward")
    else:
        L.check(lib.prtgs_precompute_transfer_backward_v(
            ctypes.byref(gs), ctypes.byref(bvh.s), ctypes.byref(p), _ptr(dP), _ptr(dV.contiguous()),
            _ptr(grads["d_means"]), _ptr(grads["d_scales"]), _ptr(grads["d_quats"]), _ptr(grads["d_opacity"]),
            _ptr(grads["d_normals"]), status.ptr() if status else None, _ptr(ws), nb, _stream()),
            "prtgs_precompute_transfer_backward_v")
    grads["_ws"] = ws
    return grads


# ------------------------------------------------------------------------------------------
# Training stage: visibility cache, view transfer (Eq. 28), pseudo-normal and normal loss (Eq. 24-25)
# ------------------------------------------------------------------------------------------
def precompute_visibility(g: GaussianTensors, bvh: Bvh, dirs: torch.Tensor, order: int,
                          t_min: float = DEFAULT_T_MIN, status: Status | None = None, walk: int = 0,
                          packet_dirs: int = 0, out: dict | None = None):
    """Visibility V [n,S] of every Gaussian along the direction set (0 where n.w <= 0) and the
    shadowed diffuse transfer P [n,C] of the same walk."""
    lib = L.load()
    dev = g.means.device
    S = int(dirs.shape[0])
    out = out or {}
    V = out.get("V") if out.get("V") is not None else torch.empty((g.n, S), dtype=torch.float32, device=dev)
    P = out.get("P") if out.get("P") is not None else torch.empty((g.n, sh_count(order)), dtype=torch.float32,
                                                                    device=dev)
    p = L.TransferParams(order, S, _ptr(dirs), float(t_min), 1.0, L.SHADOW, 0, None, 1, int(walk), int(packet_dirs))
    ws, nb = _ws(lib.prtgs_visibility_workspace_size(g.n, ctypes.byref(p)), dev)
    gs = g.struct()
    L.check(lib.prtgs_precompute_visibility(ctypes.byref(gs), ctypes.byref(bvh.s), ctypes.byref(p), _ptr(V), _ptr(P),
                                            status.ptr() if status else None, _ptr(ws), nb, _stream()),
            "prtgs_precompute_visibility")
    return {"V": V, "P": P, "_ws": ws}


def _cam3(cam_pos):
    c = np.asarray(cam_pos, dtype=np.float32).reshape(3)
    return (ctypes.c_float * 3)(*[float(x) for x in c])


def training_transfer(g: GaussianTensors, V: torch.Tensor, dirs: torch.Tensor, order: int, cam_pos,
                      out: torch.Tensor | None = None):
    """Training-stage transfer t [n,C] for the view from ``cam_pos`` (Eq. 28)."""
    lib = L.load()
    dev = g.means.device
    S = int(dirs.shape[0])
    t = out if out is not None else torch.empty((g.n, sh_count(order)), dtype=torch.float32, device=dev)
    ws, nb = _ws(lib.prtgs_training_transfer_workspace_size(order, S), dev)
    gs = g.struct()
    L.check(lib.prtgs_training_transfer(ctypes.byref(gs), order, S, _ptr(dirs), _ptr(V), _cam3(cam_pos), _ptr(t),
                                        _ptr(ws), nb, _stream()), "prtgs_training_transfer")
    return t


def training_transfer_backward(g: GaussianTensors, V: torch.Tensor, dirs: torch.Tensor, order: int, cam_pos,
                               dt: torch.Tensor):
    """d_roughness [n], d_metallic [n] from dLoss/dt [n,C] of ``training_transfer``."""
    lib = L.load()
    dev = g.means.device
    S = int(dirs.shape[0])
    dr = torch.empty(g.n, dtype=torch.float32, device=dev)
    dm = torch.empty(g.n, dtype=torch.float32, device=dev)
    dt = dt.contiguous()
    ws, nb = _ws(lib.prtgs_training_transfer_workspace_size(order, S), dev)
    gs = g.struct()
    L.check(lib.prtgs_training_transfer_backward(ctypes.byref(gs), order, S, _ptr(dirs), _ptr(V), _cam3(cam_pos),
                                                 _ptr(dt), _ptr(dr), _ptr(dm), _ptr(ws), nb, _stream()),
            "prtgs_training_transfer_backward")
    return dr, dm


def pseudo_normal(depth: torch.Tensor, cam, out: torch.Tensor | None = None):
    """Pseudo-normal map N' [3,H,W] (world space, 0 where undefined) of a depth map [H,W] (Eq. 24)."""
    lib = L.load()
    H, W = int(depth.shape[0]), int(depth.shape[1])
    Np = out if out is not None else torch.empty((3, H, W), dtype=torch.float32, device=depth.device)
    cs = camera_struct(cam)
    L.check(lib.prtgs_pseudo_normal(ctypes.byref(cs), _ptr(depth.contiguous()), _ptr(Np), _stream()),
            "prtgs_pseudo_normal")
    return Np


def normal_loss(normal: torch.Tensor, pseudo: torch.Tensor, need_grad: bool = True):
    """L = ||N - N'|| over the pixels where N' is defined (Eq. 25) as a device scalar [1], and
    dL/dN [3,H,W] (None without ``need_grad``)."""
    lib = L.load()
    H, W = int(normal.shape[1]), int(normal.shape[2])
    dev = normal.device
    loss = torch.empty(1, dtype=torch.float32, device=dev)
    dN = torch.empty((3, H, W), dtype=torch.float32, device=dev) if need_grad else None
    ws, nb = _ws(lib.prtgs_normal_loss_workspace_size(W, H), dev)
    L.check(lib.prtgs_normal_loss(W, H, _ptr(normal.contiguous()), _ptr(pseudo.contiguous()), _ptr(loss), _ptr(dN),
                                  _ptr(ws), nb, _stream()), "prtgs_normal_loss")
    return loss, dN


# ------------------------------------------------------------------------------------------
# Relight
# ------------------------------------------------------------------------------------------
def relight(T: torch.Tensor, albedo: torch.Tensor, Lsh: torch.Tensor, order: int, precision: int = L.PREC_FP32,
            glossy_ids=None, M=None, means=None, cam_pos=None, out=None, status: Status | None = None,
            tc_wait_polls: int = L.TC_WAIT_POLLS):
    """colors [k,n,3] = (albedo/pi) * (T . L_k) (Eq. 14; glossy Eq. 41). ``status`` receives
    STATUS_TIMEOUT when a tensor-core completion wait (``tc_wait_polls`` polls) gave up."""
    lib = L.load()
    n = int(T.shape[0])
    tch = 3 if T.dim() == 3 else 1
    k = int(Lsh.shape[0])
    colors = out if out is not None else torch.empty((k, n, 3), dtype=torch.float32, device=T.device)
    ng = int(glossy_ids.numel()) if glossy_ids is not None else 0
    ws, nb = _ws(lib.prtgs_relight_workspace_size(n, order, k, precision), T.device)
    L.check(lib.prtgs_relight(n, order, _ptr(T), tch, _ptr(albedo), ng, _ptr(glossy_ids), _ptr(M), _ptr(means),
                              _ptr(cam_pos), _ptr(Lsh), k, precision, _ptr(colors),
                              status.ptr() if status else None, int(tc_wait_polls), _ptr(ws), nb, _stream()),
            "prtgs_relight")
    return colors


def relight_batched(T, albedo, scene_offsets, Lsh, order, precision=L.PREC_FP32, out=None, status=None,
                    tc_wait_polls=L.TC_WAIT_POLLS):
    """Relight many scenes in one launch; Lsh [B,k,3,C] holds each scene's lights. Returns a flat
    buffer of 3kn floats holding one [k, n_b, 3] block per scene (see scene_colors)."""
    lib = L.load()
    n = int(T.shape[0])
    tch = 3 if T.dim() == 3 else 1
    B, k = int(Lsh.shape[0]), int(Lsh.shape[1])
    colors = out if out is not None else torch.empty(3 * k * n, dtype=torch.float32, device=T.device)
    L.check(lib.prtgs_relight_batched(n, order, _ptr(T), tch, _ptr(albedo), _ptr(scene_offsets), B, _ptr(Lsh), k,
                                      precision, _ptr(colors), status.ptr() if status else None,
                                      int(tc_wait_polls), _stream()), "prtgs_relight_batched")
    return colors


def scene_colors(colors_flat, k, offsets_host, b):
    """View of scene b's [k, n_b, 3] block in a prtgs_relight_batched output."""
    o0, o1 = int(offsets_host[b]), int(offsets_host[b + 1])
    return colors_flat[3 * k * o0:3 * k * o1].view(k, o1 - o0, 3)


def relight_backward(T, albedo, Lsh, order, dcolors, need_dT=False):
    lib = L.load()
    n = int(T.shape[0])
    tch = 3 if T.dim() == 3 else 1
    k = int(Lsh.shape[0])
    d_albedo = torch.empty_like(albedo)
    dT = torch.empty_like(T) if need_dT else None
    dL = torch.empty_like(Lsh)
    ws, nb = _ws(lib.prtgs_relight_backward_workspace_size(n, order, k), T.device)
    L.check(lib.prtgs_relight_backward(n, order, _ptr(T), tch, _ptr(albedo), _ptr(Lsh), k, _ptr(dcolors.contiguous()),
                                       _ptr(d_albedo), _ptr(dT), _ptr(dL), _ptr(ws), nb, _stream()),
            "prtgs_relight_backward")
    return d_albedo, dT, dL


# ------------------------------------------------------------------------------------------
# Render
# ------------------------------------------------------------------------------------------
def camera_struct(cam) -> L.Camera:
    c = L.Camera()
    rot = np.asarray(cam.rot, dtype=np.float32).reshape(-1)
    tr = np.asarray(cam.trans, dtype=np.float32).reshape(-1)
    for i in range(9):
        c.rot[i] = float(rot[i])
    for i in range(3):
        c.trans[i] = float(tr[i])
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height = int(cam.width), int(cam.height)
    c.near_plane = float(getattr(cam, "near", 0.2))
    pos = cam.position if cam.position is not None else np.zeros(3)
    for i in range(3):
        c.pos[i] = float(pos[i])
    return c


class RenderState:
    """Render state of one scene, or (n_scenes > 1) of the batched render of n_scenes scenes."""

    def __init__(self, n, width, height, max_pairs, device="cuda", n_scenes: int = 1):
        lib = L.load()
        self.n, self.width, self.height, self.max_pairs = n, width, height, int(max_pairs)
        self.n_scenes = int(n_scenes)
        self.s = L.RenderState()
        if self.n_scenes == 1:
            nbytes = lib.prtgs_render_state_bytes(n, width, height, self.max_pairs)
            self.buffer = torch.empty(int(nbytes), dtype=torch.uint8, device=device)
            L.check(lib.prtgs_render_state_init(_ptr(self.buffer), nbytes, n, width, height, self.max_pairs,
                                                ctypes.byref(self.s)), "prtgs_render_state_init")
        else:
            nbytes = lib.prtgs_render_state_bytes_batched(n, self.n_scenes, width, height, self.max_pairs)
            self.buffer = torch.empty(int(nbytes), dtype=torch.uint8, device=device)
            L.check(lib.prtgs_render_state_init_batched(_ptr(self.buffer), nbytes, n, self.n_scenes, width, height,
                                                        self.max_pairs, ctypes.byref(self.s)),
                    "prtgs_render_state_init_batched")

    def view(self, field, dtype, shape):
        off = getattr(self.s, field) - self.buffer.data_ptr()
        count = int(np.prod(shape))
        nbytes = count * torch.empty(0, dtype=dtype).element_size()
        return self.buffer[off:off + nbytes].view(dtype).view(*shape)

    def n_pairs(self) -> int:
        return int(self.view("n_pairs", torch.int32, (1,)).item())


def render(g: GaussianTensors, colors: torch.Tensor, cam, bg: torch.Tensor, state: RenderState | None = None,
           max_pairs: int | None = None, status: Status | None = None, out=None):
    """image [k,3,H,W] (Eq. 3-4)."""
    lib = L.load()
    k = int(colors.shape[0])
    if state is None:
        state = RenderState(g.n, cam.width, cam.height, max_pairs or max(16 * g.n, 1 << 16), g.means.device)
    image = out if out is not None else torch.empty((k, 3, cam.height, cam.width), dtype=torch.float32,
                                                    device=g.means.device)
    ws, nb = _ws(lib.prtgs_render_workspace_size(g.n, cam.width, cam.height, state.max_pairs), g.means.device)
    gs = g.struct()
    cs = camera_struct(cam)
    L.check(lib.prtgs_render(ctypes.byref(gs), _ptr(colors), k, ctypes.byref(cs), _ptr(bg), _ptr(image),
                             ctypes.byref(state.s), status.ptr() if status else None, _ptr(ws), nb, _stream()),
            "prtgs_render")
    state._ws = ws
    return image, state


def render_relit(g: GaussianTensors, T: torch.Tensor, Lsh: torch.Tensor, cam, order: int, bg: torch.Tensor = None,
                 precision: int = L.PREC_BF16X3, glossy_ids=None, M=None, state: RenderState | None = None,
                 max_pairs: int | None = None, status: Status | None = None, out=None,
                 tc_wait_polls: int = L.TC_WAIT_POLLS):
    """image [k,3,H,W] of every light at once in pixel space: one composite of the splats'
    (rho/pi) T (glossy: (rho/pi) M Y(v)) features, then a per-pixel contraction with the lights."""
    lib = L.load()
    dev = g.means.device
    n, k = g.n, int(Lsh.shape[0])
    tch = 3 if T.dim() == 3 else 1
    if bg is None:
        bg = torch.zeros(3, dtype=torch.float32, device=dev)
    if state is None:
        state = RenderState(n, cam.width, cam.height, max_pairs or max(16 * n, 1 << 16), dev)
    image = out if out is not None else torch.empty((k, 3, cam.height, cam.width), dtype=torch.float32, device=dev)
    ng = int(glossy_ids.numel()) if glossy_ids is not None else 0
    ws, nb = _ws(lib.prtgs_render_relit_workspace_size(n, order, cam.width, cam.height, state.max_pairs), dev)
    gs = g.struct()
    cs = camera_struct(cam)
    L.check(lib.prtgs_render_relit(ctypes.byref(gs), order, _ptr(T), tch, ng, _ptr(glossy_ids), _ptr(M), _ptr(Lsh),
                                   k, precision, ctypes.byref(cs), _ptr(bg), _ptr(image), ctypes.byref(state.s),
                                   status.ptr() if status else None, int(tc_wait_polls), _ptr(ws), nb, _stream()),
            "prtgs_render_relit")
    state._ws = ws
    return image, state


def render_geometry(g: GaussianTensors, cam, state: RenderState | None = None, max_pairs: int | None = None,
                    status: Status | None = None):
    """Depth map [H,W] and normal map [3,H,W]: composites of the splats' view-space depth and
    normal (Eq. 23, Eq. 25)."""
    lib = L.load()
    dev = g.means.device
    if state is None:
        state = RenderState(g.n, cam.width, cam.height, max_pairs or max(16 * g.n, 1 << 16), dev)
    depth = torch.empty((cam.height, cam.width), dtype=torch.float32, device=dev)
    normal = torch.empty((3, cam.height, cam.width), dtype=torch.float32, device=dev)
    ws, nb = _ws(lib.prtgs_render_geometry_workspace_size(g.n, cam.width, cam.height, state.max_pairs), dev)
    gs = g.struct()
    cs = camera_struct(cam)
    L.check(lib.prtgs_render_geometry(ctypes.byref(gs), ctypes.byref(cs), _ptr(depth), _ptr(normal),
                                      ctypes.byref(state.s), status.ptr() if status else None, _ptr(ws), nb,
                                      _stream()), "prtgs_render_geometry")
    state._ws = ws
    return depth, normal, state


def render_backward(g: GaussianTensors, colors, cam, bg, state: RenderState, dimage):
    lib = L.load()
    k = int(colors.shape[0])
    dev = g.means.device
    d_means = torch.empty_like(g.means)
    d_scales = torch.empty_like(g.scales)
    d_quats = torch.empty_like(g.quats)
    d_opacity = torch.empty_like(g.opacity)
    d_colors = torch.empty_like(colors)
    ws, nb = _ws(lib.prtgs_render_backward_workspace_size(g.n, k), dev)
    gs = g.struct()
    cs = camera_struct(cam)
    L.check(lib.prtgs_render_backward(ctypes.byref(gs), _ptr(colors), k, ctypes.byref(cs), _ptr(bg),
                                      ctypes.byref(state.s), _ptr(dimage.contiguous()), _ptr(d_means), _ptr(d_scales),
                                      _ptr(d_quats), _ptr(d_opacity), _ptr(d_colors), _ptr(ws), nb, _stream()),
            "prtgs_render_backward")
    return d_means, d_scales, d_quats, d_opacity, d_colors


def camera_array(cams):
    """Host array of prtgs_camera structs (the batched calls' per-scene cameras)."""
    arr = (L.Camera * len(cams))()
    for b, c in enumerate(cams):
        arr[b] = camera_struct(c)
    return arr


def render_batched(g: GaussianTensors, scene_offsets: torch.Tensor, colors_flat: torch.Tensor, k: int, cams,
                   bg: torch.Tensor, state: RenderState, status: Status | None = None, out=None):
    """images [B,k,3,H,W] of B scenes in one launch per stage (Eq. 3-4); colors_flat in the
    layout of relight_batched."""
    lib = L.load()
    B = len(cams)
    W, H = int(cams[0].width), int(cams[0].height)
    images = out if out is not None else torch.empty((B, k, 3, H, W), dtype=torch.float32, device=g.means.device)
    ws, nb = _ws(lib.prtgs_render_batched_workspace_size(g.n, B, W, H, state.max_pairs), g.means.device)
    gs = g.struct()
    ca = camera_array(cams)
    L.check(lib.prtgs_render_batched(ctypes.byref(gs), _ptr(scene_offsets), B, _ptr(colors_flat), k, ca, _ptr(bg),
                                     _ptr(images), ctypes.byref(state.s), status.ptr() if status else None, _ptr(ws),
                                     nb, _stream()), "prtgs_render_batched")
    state._ws = ws
    return images


def render_backward_batched(g: GaussianTensors, scene_offsets, colors_flat, k, cams, bg, state: RenderState,
                            dimages):
    """Gradients of render_batched: d_means, d_scales, d_quats, d_opacity and d_colors (batched
    colour layout)."""
    lib = L.load()
    dev = g.means.device
    out = [torch.empty_like(g.means), torch.empty_like(g.scales), torch.empty_like(g.quats),
           torch.empty_like(g.opacity), torch.empty_like(colors_flat)]
    ws, nb = _ws(lib.prtgs_render_backward_batched_workspace_size(g.n, k), dev)
    gs = g.struct()
    ca = camera_array(cams)
    L.check(lib.prtgs_render_backward_batched(ctypes.byref(gs), _ptr(scene_offsets), len(cams), _ptr(colors_flat), k,
                                              ca, _ptr(bg), ctypes.byref(state.s), _ptr(dimages.contiguous()),
                                              *(_ptr(t) for t in out), _ptr(ws), nb, _stream()),
            "prtgs_render_backward_batched")
    return tuple(out)


def l2_loss_batched(images, targets):
    """Per-scene L2 losses of images [B, ...] against targets: (losses [B], dimages)."""
    lib = L.load()
    B = int(images.shape[0])
    count = images.numel() // B
    losses = torch.empty(B, dtype=torch.float32, device=images.device)
    dimages = torch.empty_like(images)
    ws, nb = _ws(lib.prtgs_l2_loss_batched_workspace_size(count, B), images.device)
    L.check(lib.prtgs_l2_loss_batched(_ptr(images), _ptr(targets), count, B, _ptr(losses), _ptr(dimages), _ptr(ws), nb,
                                      _stream()), "prtgs_l2_loss_batched")
    return losses, dimages


def relight_backward_batched(T, albedo, scene_offsets, Lsh, order, dcolors_flat, need_dT=False):
    """Backward of relight_batched: (d_albedo [n,3], dT or None, dL [B,k,3,C])."""
    lib = L.load()
    n = int(T.shape[0])
    tch = 3 if T.dim() == 3 else 1
    B, k = int(Lsh.shape[0]), int(Lsh.shape[1])
    d_albedo = torch.empty_like(albedo)
    dT = torch.empty_like(T) if need_dT else None
    dL = torch.empty_like(Lsh)
    ws, nb = _ws(lib.prtgs_relight_backward_batched_workspace_size(n, B, order, k), T.device)
    L.check(lib.prtgs_relight_backward_batched(n, order, _ptr(T), tch, _ptr(albedo), _ptr(scene_offsets), B,
                                               _ptr(Lsh), k, _ptr(dcolors_flat), _ptr(d_albedo), _ptr(dT), _ptr(dL),
                                               _ptr(ws), nb, _stream()), "prtgs_relight_backward_batched")
    return d_albedo, dT, dL


def l2_loss(image, target):
    lib = L.load()
    count = image.numel()
    loss = torch.empty(1, dtype=torch.float32, device=image.device)
    dimage = torch.empty_like(image)
    ws, nb = _ws(lib.prtgs_l2_loss_workspace_size(count), image.device)
    L.check(lib.prtgs_l2_loss(_ptr(image), _ptr(target), count, _ptr(loss), _ptr(dimage), _ptr(ws), nb, _stream()),
            "prtgs_l2_loss")
    return loss, dimage


# ------------------------------------------------------------------------------------------
# autograd: relit splat image as a function of the Gaussians and the light
# ------------------------------------------------------------------------------------------
class RelitRender(torch.autograd.Function):
    """image = render(relight(T, albedo, L)) with the hand-written backward kernels.

    Differentiable in means, scales, quats, opacity, albedo, the light SH and T. The paper
    freezes geometry after ray tracing (Sec. 4.4), so T is usually a constant; produced by
    ShadowedTransfer instead, its gradient reaches the geometry through the transfer too.
    """

    @staticmethod
    def forward(ctx, means, scales, quats, opacity, albedo, Lsh, T, normals, cam, order, bg, max_pairs):
        g = GaussianTensors(means.contiguous(), scales.contiguous(), quats.contiguous(), opacity.contiguous(),
                            normals.contiguous(), albedo.contiguous())
        colors = relight(T.contiguous(), g.albedo, Lsh.contiguous(), order)
        image, state = render(g, colors, cam, bg, max_pairs=max_pairs)
        ctx.save_for_backward(means, scales, quats, opacity, albedo, Lsh, T, normals, colors)
        ctx.state, ctx.cam, ctx.order, ctx.bg = state, cam, order, bg
        return image

    @staticmethod
    def backward(ctx, dimage):
        means, scales, quats, opacity, albedo, Lsh, T, normals, colors = ctx.saved_tensors
        g = GaussianTensors(means.contiguous(), scales.contiguous(), quats.contiguous(), opacity.contiguous(),
                            normals.contiguous(), albedo.contiguous())
        dm, ds, dq, do, dcol = render_backward(g, colors, ctx.cam, ctx.bg, ctx.state, dimage.contiguous())
        need_dT = ctx.needs_input_grad[6]
        da, dT, dL = relight_backward(T.contiguous(), g.albedo, Lsh.contiguous(), ctx.order, dcol, need_dT=need_dT)
        return dm, ds, dq, do, da, dL, dT, None, None, None, None, None


def relit_render(means, scales, quats, opacity, albedo, Lsh, T, normals, cam, order, bg=None, max_pairs=None):
    if bg is None:
        bg = torch.zeros(3, dtype=torch.float32, device=means.device)
    return RelitRender.apply(means, scales, quats, opacity, albedo, Lsh, T, normals, cam, order, bg, max_pairs)


class ShadowedTransfer(torch.autograd.Function):
    """P = shadowed diffuse transfer of every Gaussian (Eq. 29 projected by Eq. 9) with the
    hand-written backward that recomputes the walks. Differentiable in means, scales, quats,
    opacity and normals; the hit set and the hemisphere are held fixed."""

    @staticmethod
    def forward(ctx, means, scales, quats, opacity, normals, albedo, dirs, order, t_min):
        g = GaussianTensors(means.contiguous(), scales.contiguous(), quats.contiguous(), opacity.contiguous(),
                            normals.contiguous(), albedo.contiguous())
        st = Status()
        bvh = build_bvh(g, status=st)
        P = precompute_transfer(g, bvh, dirs, order, t_min=t_min, status=st)["P"]
        ctx.g, ctx.bvh, ctx.st, ctx.dirs, ctx.order, ctx.t_min = g, bvh, st, dirs, order, t_min
        return P

    @staticmethod
    def backward(ctx, dP):
        gr = precompute_transfer_backward(ctx.g, ctx.bvh, ctx.dirs, ctx.order, dP.contiguous(), t_min=ctx.t_min,
                                          status=ctx.st)
        return (gr["d_means"], gr["d_scales"], gr["d_quats"], gr["d_opacity"], gr["d_normals"], None, None, None,
                None)


def shadowed_transfer(means, scales, quats, opacity, normals, albedo, dirs, order, t_min=DEFAULT_T_MIN):
    return ShadowedTransfer.apply(means, scales, quats, opacity, normals, albedo, dirs, order, t_min)


def bounce_backward(g: GaussianTensors, dirs: torch.Tensor, order: int, P: torch.Tensor, idx: torch.Tensor,
                    dT: torch.Tensor, n_bounces: int = 1, status: Status | None = None):
    """Backward of the self-transfer bounces (Eq. 33-35) with the index matrix fixed: from
    dT = dLoss/dT [n,3,C] to dP [n,C], d_albedo [n,3] and d_normals [n,3] (the receivers' cosines)."""
    lib = L.load()
    dev = g.means.device
    n = g.n
    C = sh_count(order)
    dP = torch.empty((n, C), dtype=torch.float32, device=dev)
    da = torch.empty((n, 3), dtype=torch.float32, device=dev)
    dn = torch.empty((n, 3), dtype=torch.float32, device=dev)
    dT = dT.contiguous()
    ws, nb = _ws(lib.prtgs_bounce_backward_workspace_size(n, order, n_bounces), dev)
    L.check(lib.prtgs_bounce_backward(n, order, int(dirs.shape[0]), _ptr(dirs), _ptr(g.normals), _ptr(g.albedo),
                                      _ptr(P), _ptr(idx), int(n_bounces), _ptr(dT), _ptr(dP), _ptr(da), _ptr(dn),
                                      status.ptr() if status else None, _ptr(ws), nb, _stream()),
            "prtgs_bounce_backward")
    return dP, da, dn


class BounceTransfer(torch.autograd.Function):
    """T = shadowed transfer with n self-transfer bounces over the index matrix (Eq. 29, Eq. 33-35)
    with the hand-written backward: the bounces' adjoint (index matrix fixed) gives dP, the albedo
    and the receivers' cosine gradients, then the transfer backward takes dP to the geometry.
    Differentiable in means, scales, quats, opacity, normals and albedo."""

    @staticmethod
    def forward(ctx, means, scales, quats, opacity, normals, albedo, dirs, order, n_bounces, t_min):
        g = GaussianTensors(means.contiguous(), scales.contiguous(), quats.contiguous(), opacity.contiguous(),
                            normals.contiguous(), albedo.contiguous())
        st = Status()
        bvh = build_bvh(g, status=st)
        out = precompute_transfer(g, bvh, dirs, order, bounce=True, n_bounces=n_bounces, t_min=t_min, status=st)
        ctx.g, ctx.bvh, ctx.st, ctx.dirs, ctx.order, ctx.t_min, ctx.nb = g, bvh, st, dirs, order, t_min, n_bounces
        ctx.P, ctx.idx = out["P"], out["idx"]
        return out["T"]

    @staticmethod
    def backward(ctx, dT):
        dP, da, dn = bounce_backward(ctx.g, ctx.dirs, ctx.order, ctx.P, ctx.idx, dT, ctx.nb, status=ctx.st)
        gr = precompute_transfer_backward(ctx.g, ctx.bvh, ctx.dirs, ctx.order, dP, t_min=ctx.t_min, status=ctx.st)
        return (gr["d_means"], gr["d_scales"], gr["d_quats"], gr["d_opacity"], gr["d_normals"] + dn, da, None, None,
                None, None)


def bounce_transfer(means, scales, quats, opacity, normals, albedo, dirs, order, n_bounces=1, t_min=DEFAULT_T_MIN):
    return BounceTransfer.apply(means, scales, quats, opacity, normals, albedo, dirs, order, n_bounces, t_min)


def glossy_backward(g: GaussianTensors, dirs: torch.Tensor, order: int, V: torch.Tensor, dM: torch.Tensor,
                    status: Status | None = None):
    """Backward of the glossy matrices (Eq. 40): dM [n_glossy,C,C] -> dV [n,S] (for
    precompute_transfer_backward's dV), d_roughness [n], d_metallic [n], d_normals [n,3]."""
    lib = L.load()
    dev = g.means.device
    n = g.n
    S = int(dirs.shape[0])
    n_glossy = int(dM.shape[0])
    f32 = dict(dtype=torch.float32, device=dev)
    dV = torch.empty((n, S), **f32)
    dr, dm, dn = torch.empty(n, **f32), torch.empty(n, **f32), torch.empty((n, 3), **f32)
    p = L.TransferParams(order, S, _ptr(dirs), float(DEFAULT_T_MIN), 1.0, L.SHADOW | L.GLOSSY, 0, None)
    ws, nb = _ws(lib.prtgs_glossy_backward_workspace_size(n, ctypes.byref(p)), dev)
    gs = g.struct()
    L.check(lib.prtgs_glossy_backward(ctypes.byref(gs), ctypes.byref(p), _ptr(V), _ptr(dM.contiguous()), n_glossy,
                                      _ptr(dV), _ptr(dr), _ptr(dm), _ptr(dn), status.ptr() if status else None,
                                      _ptr(ws), nb, _stream()), "prtgs_glossy_backward")
    return dV, dr, dm, dn


class GlossyTransfer(torch.autograd.Function):
    """(P, M): the shadowed diffuse transfer of every Gaussian (Eq. 29) and the glossy matrices of the
    glossy ones (Eq. 40), with the hand-written backward: the glossy backward turns dM into a
    visibility gradient per ray (and roughness, metallic, normal gradients), and the transfer
    backward takes dP and that visibility gradient to the geometry. Differentiable in means,
    scales, quats, opacity, normals, roughness and metallic; the glossy mask is fixed."""

    @staticmethod
    def forward(ctx, means, scales, quats, opacity, normals, roughness, metallic, glossy_mask, albedo, dirs, order,
                t_min):
        g = GaussianTensors(means.contiguous(), scales.contiguous(), quats.contiguous(), opacity.contiguous(),
                            normals.contiguous(), albedo.contiguous(), roughness.contiguous(), metallic.contiguous(),
                            glossy_mask.contiguous())
        st = Status()
        bvh = build_bvh(g, status=st)
        out = precompute_transfer(g, bvh, dirs, order, glossy=True, t_min=t_min, status=st)
        ctx.g, ctx.bvh, ctx.st, ctx.dirs, ctx.order, ctx.t_min = g, bvh, st, dirs, order, t_min
        return out["P"], out["M"]

    @staticmethod
    def backward(ctx, dP, dM):
        g = ctx.g
        V = precompute_visibility(g, ctx.bvh, ctx.dirs, ctx.order, t_min=ctx.t_min, status=ctx.st)["V"]
        if dM is None:
            dM = torch.zeros((int(g.glossy_mask.sum().item()), sh_count(ctx.order), sh_count(ctx.order)),
                             dtype=torch.float32, device=g.means.device)
        dV, dr, dm, dn = glossy_backward(g, ctx.dirs, ctx.order, V, dM, status=ctx.st)
        gr = precompute_transfer_backward(g, ctx.bvh, ctx.dirs, ctx.order, dP, t_min=ctx.t_min, status=ctx.st, dV=dV)
        return (gr["d_means"], gr["d_scales"], gr["d_quats"], gr["d_opacity"], gr["d_normals"] + dn, dr, dm, None,
                None, None, None, None)


def glossy_transfer(means, scales, quats, opacity, normals, roughness, metallic, glossy_mask, albedo, dirs, order,
                    t_min=DEFAULT_T_MIN):
    return GlossyTransfer.apply(means, scales, quats, opacity, normals, roughness, metallic, glossy_mask, albedo, dirs,
                                order, t_min)

