"""Launch-variant autotuner for libprtgs.

Each tunable call has a few launch variants that give the same result (within the stated
tolerances): the index-matrix candidate buffer of the transfer kernel (1/2/4/8 entries per
search round), the relight path (FP32 CUDA cores or the FP32-accurate 3-term BF16 split on
the tensor cores). The tuner times every variant on the actual inputs with CUDA events after
a warm-up run, keeps the fastest, and caches the choice per (device, call, shape bucket) in a
JSON file so later runs and CUDA-graph captures reuse it without timing.
"""
from __future__ import annotations

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


def time_variant(fn, repeats: int = 3) -> float:
    """Mean device time of fn() in ms (after one untimed warm-up call)."""
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(repeats):
        fn()
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1) / repeats


def choose(call: str, variants: dict, shape: dict, repeats: int = 3, force: bool = False):
    """Return the fastest variant key (cached); ``variants`` maps key -> zero-argument callable."""
    cache = _load()
    key = _key(call, **shape)
    if not force and key in cache and cache[key]["best"] in {str(v) for v in variants}:
        best = cache[key]["best"]
        return next(v for v in variants if str(v) == best)
    times = {str(v): time_variant(fn, repeats) for v, fn in variants.items()}
    best = min(times, key=times.get)
    cache[key] = {"best": best, "ms": times}
    _store(cache)
    return next(v for v in variants if str(v) == best)


def tune_transfer(g, bvh, dirs, order, bounce: bool, repeats: int = 2, force: bool = False) -> int:
    """Candidate-buffer size of the index-matrix search (only matters with bounce)."""
    from . import api

    if not bounce:
        return 0
    shape = dict(n=_bucket(g.n), S=int(dirs.shape[0]), order=order)
    variants = {kb: (lambda kb=kb: api.precompute_transfer(g, bvh, dirs, order, bounce=True, index_buffer=kb))
                for kb in (2, 4, 8)}
    return choose("transfer_index_buffer", variants, shape, repeats, force)


def tune_relight_batched(T, albedo, offsets, Lsh, order, repeats: int = 5, force: bool = False) -> int:
    """FP32 CUDA-core relight or the FP32-accurate BF16x3 tensor-core relight."""
    from . import api
    from . import _lib as L

    variants = {L.PREC_FP32: lambda: api.relight_batched(T, albedo, offsets, Lsh, order, L.PREC_FP32)}
    if T.dim() == 2 and 3 * Lsh.shape[1] <= 256:
        variants[L.PREC_BF16X3] = lambda: api.relight_batched(T, albedo, offsets, Lsh, order, L.PREC_BF16X3)
    shape = dict(n=_bucket(T.shape[0]), k=int(Lsh.shape[1]), order=order, scenes=int(Lsh.shape[0]))
    return choose("relight_precision", variants, shape, repeats, force)
