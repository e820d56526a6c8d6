"""The C-ABI library builds, loads and exports every function include/prtgs.h declares (CPU).

Also checks the host-side argument validation, which returns before any CUDA call.
"""
import ctypes
import os
import re

import pytest

from paper_2408_03538_gb300 import _lib as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "prtgs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(prtgs_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("prtgs_build_bvh", "prtgs_precompute_transfer", "prtgs_relight", "prtgs_render",
                     "prtgs_relight_backward", "prtgs_render_backward", "prtgs_relight_batched",
                     "prtgs_render_batched", "prtgs_render_backward_batched", "prtgs_relight_backward_batched"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = L.load()
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding knows every one of them
    assert set(_declared()) <= set(L.symbols())


def test_struct_sizes_match_c_layout():
    # sizes implied by include/prtgs.h on LP64
    assert ctypes.sizeof(L.Gaussians) == 8 + 9 * 8
    assert ctypes.sizeof(L.BVH) == 8 + 4 + 4 + 7 * 8
    assert ctypes.sizeof(L.TransferParams) == 4 + 4 + 8 + 4 + 4 + 4 + 4 + 8 + 4 + 4 + 4 + 4  # + tail padding
    assert ctypes.sizeof(L.Camera) == 4 * (9 + 3 + 4) + 4 * 2 + 4 + 4 * 3
    assert ctypes.sizeof(L.RenderState) == 8 + 8 + 4 * 4 + 11 * 8 + 4 + 4  # n_scenes + tail padding


def test_graph_and_autotune_argument_checks_without_gpu():
    lib = L.load()
    g = ctypes.c_void_p()
    assert lib.prtgs_graph_begin(None) == L.ERR_INVALID_ARG  # the legacy default stream cannot be captured
    assert lib.prtgs_graph_end(None, ctypes.byref(g)) == L.ERR_INVALID_ARG
    assert lib.prtgs_graph_launch(None, None) == L.ERR_INVALID_ARG
    assert lib.prtgs_graph_destroy(None) == L.OK
    best = ctypes.c_int32(-1)
    buf = ctypes.create_string_buffer(1024)
    assert lib.prtgs_autotune(99, ctypes.byref(L.TuneRelight()), 1, None, ctypes.byref(best), buf, 1024) \
        == L.ERR_INVALID_ARG
    assert lib.prtgs_autotune(L.TUNE_RELIGHT, None, 1, None, ctypes.byref(best), buf, 1024) == L.ERR_INVALID_ARG


def test_host_side_validation_without_gpu():
    lib = L.load()
    assert lib.prtgs_version() >= 10000
    assert lib.prtgs_strerror(L.ERR_WORKSPACE).decode().startswith("workspace")
    g = L.Gaussians()
    g.n = 10
    bvh = L.BVH()
    p = L.TransferParams(7, 64, ctypes.c_void_p(1), 0.0, 1.0, L.SHADOW, 0)
    # null Gaussian arrays
    assert lib.prtgs_build_bvh(ctypes.byref(g), ctypes.byref(bvh), None, None, 0, None) == L.ERR_INVALID_ARG
    # SH order outside 1..6
    fake = ctypes.c_void_p(256)
    g2 = L.Gaussians(10, fake, fake, fake, fake, fake, fake, None, None, None)
    bvh.n = 10
    assert lib.prtgs_precompute_transfer(ctypes.byref(g2), ctypes.byref(bvh), ctypes.byref(p), fake, None, None, None,
                                         0, None, None, 0, None) == L.ERR_UNSUPPORTED
    # glossy matrices whose block would need more than 227 KB of shared memory (order 6, S = 1024)
    p5 = L.TransferParams(6, 1024, fake, 0.0, 1.0, L.SHADOW | L.GLOSSY, 0)
    assert lib.prtgs_precompute_transfer(ctypes.byref(g2), ctypes.byref(bvh), ctypes.byref(p5), fake, fake, fake, None,
                                         0, None, None, 0, None) == L.ERR_UNSUPPORTED
    # ... and at the boundary: order 6 takes 608 B per direction, so S = 383 no longer fits
    p6 = L.TransferParams(6, 383, fake, 0.0, 1.0, L.SHADOW | L.GLOSSY, 0)
    assert lib.prtgs_precompute_transfer(ctypes.byref(g2), ctypes.byref(bvh), ctypes.byref(p6), fake, fake, fake, None,
                                         0, None, None, 0, None) == L.ERR_UNSUPPORTED
    # too many directions
    p2 = L.TransferParams(2, 5000, fake, 0.0, 1.0, L.SHADOW, 0)
    assert lib.prtgs_precompute_transfer(ctypes.byref(g2), ctypes.byref(bvh), ctypes.byref(p2), fake, None, None, None,
                                         0, None, None, 0, None) == L.ERR_UNSUPPORTED
    # bounce needs T and idx
    p3 = L.TransferParams(2, 64, fake, 0.0, 1.0, L.SHADOW | L.BOUNCE, 0)
    assert lib.prtgs_precompute_transfer(ctypes.byref(g2), ctypes.byref(bvh), ctypes.byref(p3), fake, None, None, None,
                                         0, None, None, 0, None) == L.ERR_INVALID_ARG
    # workspace too small
    need = lib.prtgs_build_bvh_workspace_size(10, 1)
    assert need > 0
    bvh2 = L.BVH(10, 1, 0, fake, fake, fake, fake, fake, fake, fake)
    assert lib.prtgs_build_bvh(ctypes.byref(g2), ctypes.byref(bvh2), None, fake, need - 1, None) == L.ERR_WORKSPACE
    # misaligned workspace
    assert lib.prtgs_build_bvh(ctypes.byref(g2), ctypes.byref(bvh2), None, ctypes.c_void_p(264), need,
                               None) == L.ERR_WORKSPACE
    # relight: bad channel count and precision
    assert lib.prtgs_relight(10, 2, fake, 2, fake, 0, None, None, None, None, fake, 1, 0, fake, None,
                             L.TC_WAIT_POLLS, None, 0, None) == L.ERR_SHAPE
    assert lib.prtgs_relight(10, 2, fake, 1, fake, 0, None, None, None, None, fake, 1, 7, fake, None,
                             L.TC_WAIT_POLLS, None, 0, None) == L.ERR_INVALID_ARG
    # BVH layout: too many scenes
    out = L.BVH()
    assert lib.prtgs_bvh_init(fake, 1 << 20, 10, 200, fake, ctypes.byref(out)) == L.ERR_UNSUPPORTED


def test_layout_queries_are_consistent():
    lib = L.load()
    a = lib.prtgs_bvh_bytes(1000, 1)
    b = lib.prtgs_bvh_bytes(2000, 1)
    assert 0 < a < b
    assert lib.prtgs_render_state_bytes(100, 64, 48, 1000) > lib.prtgs_render_state_bytes(100, 64, 48, 10)
    # empty problems need no workspace and succeed without touching the GPU
    g0 = L.Gaussians()
    bvh0 = L.BVH(0, 1, 0, None, None, None, None, None, None, ctypes.c_void_p(256))
    assert lib.prtgs_build_bvh(ctypes.byref(g0), ctypes.byref(bvh0), None, None, 0, None) == L.OK


def test_training_calls_validate_on_the_host():
    """The visibility cache, training transfer, pseudo-normal and normal-loss entry points reject
    bad arguments before any device work."""
    lib = L.load()
    fake = ctypes.c_void_p(256)
    g = L.Gaussians(10, fake, fake, fake, fake, fake, fake, fake, fake, None)
    bvh = L.BVH(10, 1, 0, fake, fake, fake, fake, fake, fake, fake)
    cam = (ctypes.c_float * 3)(0.0, -3.0, 1.0)
    # visibility: only PRTGS_SHADOW, P and V required
    pb = L.TransferParams(3, 64, fake, 0.0, 1.0, L.SHADOW | L.BOUNCE, 0)
    assert lib.prtgs_precompute_visibility(ctypes.byref(g), ctypes.byref(bvh), ctypes.byref(pb), fake, fake, None,
                                           None, 0, None) == L.ERR_UNSUPPORTED
    ps = L.TransferParams(3, 64, fake, 0.0, 1.0, L.SHADOW, 0)
    assert lib.prtgs_precompute_visibility(ctypes.byref(g), ctypes.byref(bvh), ctypes.byref(ps), None, fake, None,
                                           None, 0, None) == L.ERR_INVALID_ARG
    assert lib.prtgs_precompute_visibility(ctypes.byref(g), ctypes.byref(bvh), ctypes.byref(ps), fake, fake, None,
                                           None, 0, None) == L.ERR_WORKSPACE
    assert lib.prtgs_visibility_workspace_size(10, ctypes.byref(ps)) > lib.prtgs_transfer_workspace_size(
        10, 0, ctypes.byref(ps))  # the identity slots
    # training transfer: order 1..6, directions 1..1024, camera, BRDF parameters, workspace
    need = lib.prtgs_training_transfer_workspace_size(3, 64)
    assert need >= 64 * 16 * 4 and lib.prtgs_training_transfer_workspace_size(7, 64) == 0
    assert lib.prtgs_training_transfer(ctypes.byref(g), 7, 64, fake, fake, cam, fake, fake, need, None) == \
        L.ERR_UNSUPPORTED
    assert lib.prtgs_training_transfer(ctypes.byref(g), 3, 2000, fake, fake, cam, fake, fake, need, None) == \
        L.ERR_UNSUPPORTED
    assert lib.prtgs_training_transfer(ctypes.byref(g), 3, 64, fake, fake, None, fake, fake, need, None) == \
        L.ERR_INVALID_ARG
    nan_cam = (ctypes.c_float * 3)(0.0, float("nan"), 1.0)
    assert lib.prtgs_training_transfer(ctypes.byref(g), 3, 64, fake, fake, nan_cam, fake, fake, need, None) == \
        L.ERR_INVALID_ARG
    g_nobrdf = L.Gaussians(10, fake, fake, fake, fake, fake, fake, None, None, None)
    assert lib.prtgs_training_transfer(ctypes.byref(g_nobrdf), 3, 64, fake, fake, cam, fake, fake, need, None) == \
        L.ERR_INVALID_ARG
    assert lib.prtgs_training_transfer(ctypes.byref(g), 3, 64, fake, fake, cam, fake, fake, need - 1, None) == \
        L.ERR_WORKSPACE
    assert lib.prtgs_training_transfer_backward(ctypes.byref(g), 3, 64, fake, fake, cam, fake, None, fake, fake,
                                                need, None) == L.ERR_INVALID_ARG
    # pseudo-normal and normal loss
    c = L.Camera()
    c.width, c.height, c.fx, c.fy = 8, 6, 0.0, 10.0
    assert lib.prtgs_pseudo_normal(ctypes.byref(c), fake, fake, None) == L.ERR_INVALID_ARG
    c.fx = 10.0
    assert lib.prtgs_pseudo_normal(ctypes.byref(c), None, fake, None) == L.ERR_INVALID_ARG
    c.width = 0
    assert lib.prtgs_pseudo_normal(ctypes.byref(c), None, None, None) == L.OK  # empty image: nothing to do
    assert lib.prtgs_normal_loss(8, 6, fake, fake, None, None, fake, 1 << 20, None) == L.ERR_INVALID_ARG
    nl = lib.prtgs_normal_loss_workspace_size(1920, 1080)
    assert nl >= 8 and lib.prtgs_normal_loss(1920, 1080, fake, fake, fake, None, fake, nl - 1, None) == \
        L.ERR_WORKSPACE
