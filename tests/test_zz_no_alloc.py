"""The allocation-free relight backward against the regular entry point (GPU).

prtgs_relight_backward_noalloc is for callers that cannot give the library device memory
(a host application owning all device allocations through its own pool, or a loop that
must not call cudaMalloc). It keeps its scratch in a fixed array in the library's device
memory; this file runs last so that a failure here never hides the rest of the suite.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2408_03538_gb300 import _lib as L
from paper_2408_03538_gb300 import api

pytestmark = pytest.mark.gpu


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _case(seed, n, tch, k, order=3):
    g = torch.Generator(device="cpu").manual_seed(seed)
    C = (order + 1) ** 2
    T = torch.randn((n, C) if tch == 1 else (n, 3, C), generator=g).cuda()
    alb = torch.rand((n, 3), generator=g).cuda()
    Lsh = torch.randn((k, 3, C), generator=g).cuda()
    dcol = torch.randn((k, n, 3), generator=g).cuda()
    return T, alb, Lsh, dcol


def _noalloc(T, alb, Lsh, dcol, order, need_dT=True):
    lib = L.load()
    n, k = T.shape[0], Lsh.shape[0]
    tch = 3 if T.dim() == 3 else 1
    da = torch.full_like(alb, float("nan"))
    dT = torch.full_like(T, float("nan")) if need_dT else None
    dL = torch.full_like(Lsh, float("nan"))
    rc = lib.prtgs_relight_backward_noalloc(n, order, _p(T), tch, _p(alb), _p(Lsh), k, _p(dcol), _p(da), _p(dT),
                                            _p(dL), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == L.OK, rc
    return da, dT, dL


def _rel(a, b):
    return float((a - b).norm() / b.norm().clamp_min(1e-30))


def test_noalloc_matches_regular_entry_point_twice_in_a_row():
    order = 3
    # two consecutive calls with different sizes and inputs: the shared scratch keeps the
    # first call's partial sums, which the second call must not pick up
    for seed, n, tch, k in ((1, 70001, 3, 2), (2, 5003, 1, 5)):
        T, alb, Lsh, dcol = _case(seed, n, tch, k, order)
        da, dT, dL = _noalloc(T, alb, Lsh, dcol, order)
        ra, rT, rL = api.relight_backward(T, alb, Lsh, order, dcol, need_dT=True)
        torch.cuda.synchronize()
        assert _rel(da, ra) < 1e-5 and _rel(dT, rT) < 1e-5 and _rel(dL, rL) < 1e-5


def test_noalloc_rejects_problems_beyond_its_scratch():
    lib = L.load()
    cap = lib.prtgs_relight_backward_noalloc_max_bytes()
    assert cap == 1 << 20
    fake = ctypes.c_void_p(256)
    # ceil(n/2048) * k * 48 floats must fit: n = 2^24, k = 64 does not
    rc = lib.prtgs_relight_backward_noalloc(1 << 24, 3, fake, 1, fake, fake, 64, fake, fake, None, fake, None)
    assert rc == L.ERR_UNSUPPORTED
