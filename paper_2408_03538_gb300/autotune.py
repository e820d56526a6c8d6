"""Autotuner cache for libprtgs launch variants.

The timing itself is the library's: prtgs_autotune (C) runs every launch variant of a call on
the caller's inputs with CUDA events and returns a JSON report. This module keeps those reports
in a JSON file keyed by (device, call, shape bucket), so later runs and CUDA-graph captures reuse
the choice without timing again:
  * transfer: the warp-packet walk with its directions per work item (the work tile: 32
    receivers x packet_dirs directions), 1..32, or the per-ray walk (reported as 0);
  * relight: FP32 CUDA cores or the FP32-accurate 3-term BF16 split on the tensor cores.
"""
from __future__ import annotations

import ctypes
import json
import math
import os

import torch

_DEFAULT_CACHE = os.path.join(os.environ.get("XDG_CACHE_HOME", os.path.expanduser("~/.cache")), "prtgs",
                              "autotune.json")


def cache_path() -> str:
    return os.environ.get("PRTGS_TUNE_CACHE", _DEFAULT_CACHE)


def _load():
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(d):
    p = cache_path()
    try:
        os.makedirs(os.path.dirname(p), exist_ok=True)
        tmp = p + ".tmp"
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, p)
    except OSError:
        pass  # a read-only home only costs re-tuning


def _bucket(x: int) -> int:
    """Shape bucket: the next power of two (so nearby sizes share a tuning result)."""
    return 1 << max(0, math.ceil(math.log2(max(1, x))))


def _key(call: str, **shape) -> str:
    dev = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    return dev + "|" + call + "|" + ",".join(f"{k}={v}" for k, v in sorted(shape.items()))


def _run(kernel_id: int, args, repeats: int) -> dict:
    """prtgs_autotune on the current stream: the JSON report (with "best")."""
    from . import _lib as L
    from .api import _stream

    lib = L.load()
    best = ctypes.c_int32(-1)
    buf = ctypes.create_string_buffer(4096)
    L.check(lib.prtgs_autotune(kernel_id, ctypes.byref(args), repeats, _stream(), ctypes.byref(best), buf, 4096),
            "prtgs_autotune")
    rep = json.loads(buf.value.decode())
    assert rep["best"] == best.value
    return rep


def _cached(call: str, shape: dict, measure, force: bool):
    cache = _load()
    key = _key(call, **shape)
    if not force and key in cache:
        return cache[key]["best"]
    rep = measure()
    cache[key] = rep
    _store(cache)
    return rep["best"]


def tune_transfer(g, bvh, dirs, order, bounce: bool, repeats: int = 1, force: bool = False) -> int:
    """The fastest transfer walk for this shape: packet_dirs of the packet walk, or 0 for the
    per-ray walk (walk=1)."""
    from . import _lib as L
    from . import api

    S = int(dirs.shape[0])
    C = (order + 1) ** 2
    flags = L.SHADOW | (L.BOUNCE if bounce else 0)
    shape = dict(n=_bucket(g.n), S=S, order=order, bounce=int(bounce))

    def measure():
        dev = g.means.device
        P = torch.empty((g.n, C), dtype=torch.float32, device=dev)
        T = torch.empty((g.n, 3, C), dtype=torch.float32, device=dev) if bounce else None
        idx = torch.empty((g.n, S), dtype=torch.int32, device=dev) if bounce else None
        p = L.TransferParams(order, S, api._ptr(dirs), float(api.DEFAULT_T_MIN), 1.0, flags, 0, None, 1, 1, 0)
        lib = L.load()
        need = lib.prtgs_transfer_workspace_size(g.n, 0, ctypes.byref(p))  # the per-ray walk's
        p.walk = 0
        need = max(need, lib.prtgs_transfer_workspace_size(g.n, 0, ctypes.byref(p)))  # and the packet walk's
        ws, nb = api._ws(need, dev)
        gs = g.struct()
        args = L.TuneTransfer(ctypes.addressof(gs), ctypes.addressof(bvh.s), p, api._ptr(P), api._ptr(T),
                              api._ptr(idx), None, 0, None, api._ptr(ws), nb)
        return _run(L.TUNE_TRANSFER, args, repeats)

    return int(_cached("transfer_packet_dirs", shape, measure, force))


def tune_relight_batched(T, albedo, offsets, Lsh, order, repeats: int = 5, force: bool = False) -> int:
    """FP32 CUDA-core relight or the FP32-accurate BF16x3 tensor-core relight."""
    from . import _lib as L
    from . import api

    n = int(T.shape[0])
    tch = 3 if T.dim() == 3 else 1
    B, k = int(Lsh.shape[0]), int(Lsh.shape[1])
    shape = dict(n=_bucket(n), k=k, order=order, scenes=B, t_channels=tch)

    def measure():
        colors = torch.empty(3 * k * n, dtype=torch.float32, device=T.device)
        args = L.TuneRelight(n, order, tch, api._ptr(T), api._ptr(albedo), api._ptr(offsets), B, k, api._ptr(Lsh),
                             api._ptr(colors), None)
        return _run(L.TUNE_RELIGHT, args, repeats)

    return int(_cached("relight_precision", shape, measure, force))
