"""The tensor-core relight's bounded completion wait: when it gives up, the call reports
PRTGS_STATUS_TIMEOUT, the affected outputs are NaN, and the GPU stays usable (the CTA drained its
MMA chain before reusing or freeing its shared and tensor memory), so the next call with the
default limit is correct.

The failure is made with tc_wait_polls = 0: the first wait of every CTA gives up without polling,
while the tensor cores themselves finish normally (the drain's second wait sees them complete).
Nothing here faults, traps or hangs the GPU.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import render as OR
from paper_2408_03538_gb300 import _lib as L, api, scenes as S

pytestmark = pytest.mark.gpu


def _cuda(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype).contiguous()


@pytest.mark.parametrize("tch", [1, 3])
def test_relight_wait_timeout_then_recovery(tch):
    rng = np.random.default_rng(90 + tch)
    n, C, k = 3001, 16, 8
    T = rng.standard_normal((n, C) if tch == 1 else (n, 3, C)).astype(np.float32)
    alb = rng.uniform(0, 1, (n, 3)).astype(np.float32)
    Lsh = rng.standard_normal((k, 3, C)).astype(np.float32)
    Tg, ag, Lg = _cuda(T), _cuda(alb), _cuda(Lsh)
    st = api.Status()
    col = api.relight(Tg, ag, Lg, 3, precision=L.PREC_BF16X3, status=st, tc_wait_polls=0)
    torch.cuda.synchronize()
    assert st.read() & L.STATUS_TIMEOUT
    assert torch.isnan(col).all()  # every CTA gave up on its first tile, hence on all of them
    st2 = api.Status()
    col2 = api.relight(Tg, ag, Lg, 3, precision=L.PREC_BF16X3, status=st2).cpu().numpy()
    assert st2.read() == 0
    ref = oracle.relight(T, alb, Lsh)
    err = oracle.norm_err(col2.transpose(1, 0, 2), ref.transpose(1, 0, 2), 1e-6)
    assert err.max() < 1e-4


def test_pixel_relight_wait_timeout_then_recovery():
    sc = S.surface_scene(800, 91)
    sc.means *= 0.5
    rng = np.random.default_rng(91)
    n, C, k = sc.n, 16, 4
    T = (rng.standard_normal((n, 3, C)) * 0.3).astype(np.float32)
    T[..., 0] += 1.2
    Lsh = S.env_lights(k, 3, 92)
    cam = S.look_at_camera((0, -4.0, 2.0), (0, 0, 0.4), 45, 64, 48)
    g = api.GaussianTensors.from_scene(sc)
    st = api.Status()
    img, _ = api.render_relit(g, _cuda(T), _cuda(Lsh), cam, 3, precision=L.PREC_BF16X3, status=st, tc_wait_polls=0)
    torch.cuda.synchronize()
    assert st.read() & L.STATUS_TIMEOUT
    assert torch.isnan(img).all()
    st2 = api.Status()
    img2, _ = api.render_relit(g, _cuda(T), _cuda(Lsh), cam, 3, precision=L.PREC_BF16X3, status=st2)
    torch.cuda.synchronize()
    assert st2.read() == 0
    col = oracle.relight(T, sc.albedo, Lsh)
    t = lambda a: torch.as_tensor(np.asarray(a, np.float64))
    ref = OR.render(t(sc.means), t(sc.scales), t(sc.quats), t(sc.opacity), t(col), cam).numpy()
    img2 = img2.cpu().numpy()
    peak = float(np.abs(ref).max())
    for l in range(k):
        assert OR.psnr(img2[l], ref[l], peak=peak) >= 50.0, l
