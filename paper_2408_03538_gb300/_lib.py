"""ctypes loader for libprtgs.so: struct mirrors of include/prtgs.h and the function table.

Argument marshalling only. Every computation happens in the CUDA library; there is no
CPU fallback. Loading fails loudly when the library cannot be built or found.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libprtgs.so")

c_int32, c_int64, c_uint32, c_float, c_size_t, c_void_p = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                                            ctypes.c_float, ctypes.c_size_t, ctypes.c_void_p)

# status codes and flags (include/prtgs.h)
OK, ERR_INVALID_ARG, ERR_SHAPE, ERR_UNSUPPORTED, ERR_WORKSPACE, ERR_CUDA = 0, -1, -2, -3, -4, -5
STATUS_NONFINITE, STATUS_STACK_OVERFLOW, STATUS_CAPACITY, STATUS_BAD_INDEX, STATUS_TIMEOUT = 1, 2, 4, 8, 16
TC_WAIT_POLLS = 1 << 26
SHADOW, BOUNCE, GLOSSY = 1, 2, 4
PREC_FP32, PREC_BF16X3, PREC_BF16 = 0, 1, 2


class Gaussians(ctypes.Structure):
    _fields_ = [("n", c_int64), ("means", c_void_p), ("scales", c_void_p), ("quats", c_void_p),
                ("opacity", c_void_p), ("normals", c_void_p), ("albedo", c_void_p), ("roughness", c_void_p),
                ("metallic", c_void_p), ("glossy_mask", c_void_p)]


class BVH(ctypes.Structure):
    _fields_ = [("n", c_int64), ("n_scenes", c_int32), ("reserved", c_int32), ("keys", c_void_p),
                ("order", c_void_p), ("nodes", c_void_p), ("records", c_void_p), ("leaf_parent", c_void_p),
                ("roots", c_void_p), ("scene_offsets", c_void_p)]


class TransferParams(ctypes.Structure):
    _fields_ = [("sh_order", c_int32), ("n_dirs", c_int32), ("dirs", c_void_p), ("t_min", c_float),
                ("same_surface_t", c_float), ("flags", c_uint32), ("index_buffer", c_int32), ("stats", c_void_p),
                ("n_bounces", c_int32), ("walk", c_int32), ("packet_dirs", c_int32)]


class TuneTransfer(ctypes.Structure):
    _fields_ = [("g", ctypes.c_void_p), ("bvh", ctypes.c_void_p), ("params", TransferParams), ("P", c_void_p),
                ("T", c_void_p), ("idx", c_void_p), ("M", c_void_p), ("n_glossy", c_int64), ("status", c_void_p),
                ("workspace", c_void_p), ("workspace_bytes", c_size_t)]


class TuneRelight(ctypes.Structure):
    _fields_ = [("n", c_int64), ("sh_order", c_int32), ("t_channels", c_int32), ("T", c_void_p),
                ("albedo", c_void_p), ("scene_offsets", c_void_p), ("n_scenes", c_int32), ("k", c_int32),
                ("L", c_void_p), ("colors", c_void_p), ("status", c_void_p)]


TUNE_TRANSFER, TUNE_RELIGHT = 1, 2


class Camera(ctypes.Structure):
    _fields_ = [("rot", c_float * 9), ("trans", c_float * 3), ("fx", c_float), ("fy", c_float), ("cx", c_float),
                ("cy", c_float), ("width", c_int32), ("height", c_int32), ("near_plane", c_float),
                ("pos", c_float * 3)]


class RenderState(ctypes.Structure):
    _fields_ = [("n", c_int64), ("max_pairs", c_int64), ("width", c_int32), ("height", c_int32),
                ("tiles_x", c_int32), ("tiles_y", c_int32), ("mean2d", c_void_p), ("conic_op", c_void_p),
                ("depth", c_void_p), ("radius", c_void_p), ("tiles_touched", c_void_p), ("pair_keys", c_void_p),
                ("pair_ids", c_void_p), ("ranges", c_void_p), ("final_T", c_void_p), ("n_contrib", c_void_p),
                ("n_pairs", c_void_p), ("n_scenes", c_int32)]


P = ctypes.POINTER
_SIGS = {
    "prtgs_version": (c_int32, []),
    "prtgs_launch_count": (ctypes.c_ulonglong, []),
    "prtgs_strerror": (ctypes.c_char_p, [c_int32]),
    "prtgs_read_status": (c_int32, [c_void_p, c_void_p]),
    "prtgs_bvh_bytes": (c_size_t, [c_int64, c_int32]),
    "prtgs_bvh_init": (c_int32, [c_void_p, c_size_t, c_int64, c_int32, c_void_p, P(BVH)]),
    "prtgs_build_bvh_workspace_size": (c_size_t, [c_int64, c_int32]),
    "prtgs_build_bvh": (c_int32, [P(Gaussians), P(BVH), c_void_p, c_void_p, c_size_t, c_void_p]),
    "prtgs_transfer_workspace_size": (c_size_t, [c_int64, c_int64, P(TransferParams)]),
    "prtgs_precompute_transfer": (c_int32, [P(Gaussians), P(BVH), P(TransferParams), c_void_p, c_void_p, c_void_p,
                                            c_void_p, c_int64, c_void_p, c_void_p, c_size_t, c_void_p]),
    "prtgs_transfer_backward_workspace_size": (c_size_t, [c_int64, P(TransferParams)]),
    "prtgs_precompute_transfer_backward": (c_int32, [P(Gaussians), P(BVH), P(TransferParams), c_void_p, c_void_p,
                                                     c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                                     c_size_t, c_void_p]),
    "prtgs_render_relit_workspace_size": (c_size_t, [c_int64, c_int32, c_int32, c_int32, c_int64]),
    "prtgs_render_relit": (c_int32, [P(Gaussians), c_int32, c_void_p, c_int32, c_int64, c_void_p, c_void_p,
                                     c_void_p, c_int32, c_int32, P(Camera), c_void_p, c_void_p, P(RenderState),
                                     c_void_p, c_uint32, c_void_p, c_size_t, c_void_p]),
    "prtgs_render_geometry_workspace_size": (c_size_t, [c_int64, c_int32, c_int32, c_int64]),
    "prtgs_render_geometry": (c_int32, [P(Gaussians), P(Camera), c_void_p, c_void_p, P(RenderState), c_void_p,
                                        c_void_p, c_size_t, c_void_p]),
    "prtgs_relight_workspace_size": (c_size_t, [c_int64, c_int32, c_int32, c_int32]),
    "prtgs_relight": (c_int32, [c_int64, c_int32, c_void_p, c_int32, c_void_p, c_int64, c_void_p, c_void_p,
                                c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_void_p, c_void_p, c_uint32,
                                c_void_p, c_size_t, c_void_p]),
    "prtgs_relight_batched": (c_int32, [c_int64, c_int32, c_void_p, c_int32, c_void_p, c_void_p, c_int32, c_void_p,
                                        c_int32, c_int32, c_void_p, c_void_p, c_uint32, c_void_p]),
    "prtgs_relight_backward_workspace_size": (c_size_t, [c_int64, c_int32, c_int32]),
    "prtgs_relight_backward": (c_int32, [c_int64, c_int32, c_void_p, c_int32, c_void_p, c_void_p, c_int32,
                                         c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "prtgs_relight_backward_noalloc_max_bytes": (c_size_t, []),
    "prtgs_relight_backward_noalloc": (c_int32, [c_int64, c_int32, c_void_p, c_int32, c_void_p, c_void_p, c_int32,
                                                 c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "prtgs_render_state_bytes": (c_size_t, [c_int64, c_int32, c_int32, c_int64]),
    "prtgs_render_state_init": (c_int32, [c_void_p, c_size_t, c_int64, c_int32, c_int32, c_int64, P(RenderState)]),
    "prtgs_render_workspace_size": (c_size_t, [c_int64, c_int32, c_int32, c_int64]),
    "prtgs_render": (c_int32, [P(Gaussians), c_void_p, c_int32, P(Camera), c_void_p, c_void_p, P(RenderState),
                               c_void_p, c_void_p, c_size_t, c_void_p]),
    "prtgs_render_backward_workspace_size": (c_size_t, [c_int64, c_int32]),
    "prtgs_render_backward": (c_int32, [P(Gaussians), c_void_p, c_int32, P(Camera), c_void_p, P(RenderState),
                                        c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                        c_size_t, c_void_p]),
    "prtgs_render_state_bytes_batched": (c_size_t, [c_int64, c_int32, c_int32, c_int32, c_int64]),
    "prtgs_render_state_init_batched": (c_int32, [c_void_p, c_size_t, c_int64, c_int32, c_int32, c_int32, c_int64,
                                                  P(RenderState)]),
    "prtgs_render_batched_workspace_size": (c_size_t, [c_int64, c_int32, c_int32, c_int32, c_int64]),
    "prtgs_render_batched": (c_int32, [P(Gaussians), c_void_p, c_int32, c_void_p, c_int32, c_void_p, c_void_p,
                                       c_void_p, P(RenderState), c_void_p, c_void_p, c_size_t, c_void_p]),
    "prtgs_render_backward_batched_workspace_size": (c_size_t, [c_int64, c_int32]),
    "prtgs_render_backward_batched": (c_int32, [P(Gaussians), c_void_p, c_int32, c_void_p, c_int32, c_void_p,
                                                c_void_p, P(RenderState), c_void_p, c_void_p, c_void_p, c_void_p,
                                                c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "prtgs_l2_loss_batched_workspace_size": (c_size_t, [c_int64, c_int32]),
    "prtgs_l2_loss_batched": (c_int32, [c_void_p, c_void_p, c_int64, c_int32, c_void_p, c_void_p, c_void_p, c_size_t,
                                        c_void_p]),
    "prtgs_relight_backward_batched_workspace_size": (c_size_t, [c_int64, c_int32, c_int32, c_int32]),
    "prtgs_relight_backward_batched": (c_int32, [c_int64, c_int32, c_void_p, c_int32, c_void_p, c_void_p, c_int32,
                                                 c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                                 c_size_t, c_void_p]),
    "prtgs_glossy_backward_workspace_size": (c_size_t, [c_int64, P(TransferParams)]),
    "prtgs_glossy_backward": (c_int32, [P(Gaussians), P(TransferParams), c_void_p, c_void_p, c_int64, c_void_p,
                                        c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "prtgs_precompute_transfer_backward_v": (c_int32, [P(Gaussians), P(BVH), P(TransferParams), c_void_p, c_void_p,
                                                       c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                                       c_void_p, c_size_t, c_void_p]),
    "prtgs_bounce_backward_workspace_size": (c_size_t, [c_int64, c_int32, c_int32]),
    "prtgs_bounce_backward": (c_int32, [c_int64, c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                        c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t,
                                        c_void_p]),
    "prtgs_visibility_workspace_size": (c_size_t, [c_int64, P(TransferParams)]),
    "prtgs_precompute_visibility": (c_int32, [P(Gaussians), P(BVH), P(TransferParams), c_void_p, c_void_p, c_void_p,
                                              c_void_p, c_size_t, c_void_p]),
    "prtgs_training_transfer_workspace_size": (c_size_t, [c_int32, c_int32]),
    "prtgs_training_transfer": (c_int32, [P(Gaussians), c_int32, c_int32, c_void_p, c_void_p, P(c_float), c_void_p,
                                          c_void_p, c_size_t, c_void_p]),
    "prtgs_training_transfer_backward": (c_int32, [P(Gaussians), c_int32, c_int32, c_void_p, c_void_p, P(c_float),
                                                   c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "prtgs_pseudo_normal": (c_int32, [P(Camera), c_void_p, c_void_p, c_void_p]),
    "prtgs_normal_loss_workspace_size": (c_size_t, [c_int32, c_int32]),
    "prtgs_normal_loss": (c_int32, [c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t,
                                    c_void_p]),
    "prtgs_autotune": (c_int32, [c_int32, c_void_p, c_int32, c_void_p, P(c_int32), ctypes.c_char_p, c_size_t]),
    "prtgs_graph_begin": (c_int32, [c_void_p]),
    "prtgs_graph_end": (c_int32, [c_void_p, P(c_void_p)]),
    "prtgs_graph_launch": (c_int32, [c_void_p, c_void_p]),
    "prtgs_graph_destroy": (c_int32, [c_void_p]),
    "prtgs_l2_loss_workspace_size": (c_size_t, [c_int64]),
    "prtgs_l2_loss": (c_int32, [c_void_p, c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
}

_lib = None


def load(build_if_missing: bool = True):
    """Load libprtgs.so (building it with nvcc first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        from . import build as _build

        _build.build()
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libprtgs.so not found at {LIB_PATH}; run paper_2408_03538_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def symbols():
    return list(_SIGS)


class PrtgsError(RuntimeError):
    pass


def check(rc: int, what: str):
    if rc != OK:
        msg = load().prtgs_strerror(rc).decode()
        raise PrtgsError(f"{what}: {msg} ({rc})")
