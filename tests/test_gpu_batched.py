"""Batched scenes: one BVH + one persistent transfer launch over all scenes, one relight launch
with per-scene lights, graph capture and replay (GPU)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2408_03538_gb300 import api, autotune, batched, scenes as S

pytestmark = pytest.mark.gpu


def _scenes(sizes, seed=5):
    return [S.isotropic_scene(n, seed * 1000 + i) for i, n in enumerate(sizes)]


def test_batched_transfer_equals_per_scene():
    sizes = [3000, 1, 0, 700, 12345]
    parts = _scenes(sizes)
    merged, offs = S.concat_scenes(parts)
    dirs = torch.from_numpy(S.direction_set(128, 3)).cuda()
    g = api.GaussianTensors.from_scene(merged)
    bvh = api.build_bvh(g, torch.from_numpy(offs).cuda())
    P = api.precompute_transfer(g, bvh, dirs, 3)["P"].cpu().numpy()
    for b, sc in enumerate(parts):
        if sc.n == 0:
            continue
        gb = api.GaussianTensors.from_scene(sc)
        Pb = api.precompute_transfer(gb, api.build_bvh(gb), dirs, 3)["P"].cpu().numpy()
        np.testing.assert_allclose(P[offs[b]:offs[b + 1]], Pb, rtol=0, atol=1e-6)
    # and one scene against the oracle (sampled receivers)
    recv = np.arange(offs[3], offs[4], 37)
    ref = oracle.transfer(merged.subset(np.arange(offs[3], offs[4])), dirs.cpu().numpy(), 3, recv - offs[3])
    err = np.linalg.norm(P[recv] - ref["P"], axis=1)
    lim = 1e-4 * np.maximum(np.linalg.norm(ref["P"], axis=1), 1e-3 * oracle.unoccluded_norm(3)) + ref["allow_P"]
    assert np.all(err <= lim)


@pytest.mark.parametrize("precision", [0, 1])
def test_relight_batched_equals_per_scene(precision):
    rng = np.random.default_rng(3)
    sizes = [129, 1000, 1, 257, 0, 64]
    offs = np.zeros(len(sizes) + 1, np.int64)
    offs[1:] = np.cumsum(sizes)
    n, C, k = int(offs[-1]), 16, 8
    T = torch.from_numpy(rng.standard_normal((n, C)).astype(np.float32)).cuda()
    alb = torch.from_numpy(rng.uniform(0, 1, (n, 3)).astype(np.float32)).cuda()
    Lsh = torch.from_numpy(rng.standard_normal((len(sizes), k, 3, C)).astype(np.float32)).cuda()
    flat = api.relight_batched(T, alb, torch.from_numpy(offs).cuda(), Lsh, 3, precision)
    for b in range(len(sizes)):
        if sizes[b] == 0:
            continue
        got = api.scene_colors(flat, k, offs, b).cpu().numpy()
        ref = oracle.relight(T[offs[b]:offs[b + 1]].cpu().numpy(), alb[offs[b]:offs[b + 1]].cpu().numpy(),
                             Lsh[b].cpu().numpy())
        err = oracle.norm_err(got.transpose(1, 0, 2), ref.transpose(1, 0, 2), 1e-3)
        assert err.max() < 1e-4


def test_graph_replay_matches_eager_and_autotuner_caches(tmp_path, monkeypatch):
    monkeypatch.setenv("PRTGS_TUNE_CACHE", str(tmp_path / "tune.json"))
    sizes = [2000, 500, 4000]
    parts = _scenes(sizes, 9)
    lights = np.stack([S.env_lights(4, 3, 50 + b) for b in range(len(sizes))])
    cams = [S.look_at_camera((0, -3.5, 1.5), (0, 0, 0), 50, 160, 96) for _ in sizes]
    pipe = batched.BatchedPipeline(parts, S.direction_set(64, 4), 3, lights, cams)
    assert (tmp_path / "tune.json").exists()
    eager = pipe.step()
    imgs = [im.clone() for im in pipe.images]
    dL = [d.clone() for d in eager["dL"]]
    g_means = [g[0].clone() for g in eager["grads"]]
    pipe.capture()
    # perturb the outputs, replay, and compare with the eager pass
    for im in pipe.images:
        im.fill_(-1)
    cap = pipe.replay()
    torch.cuda.synchronize()
    for b in range(len(sizes)):
        torch.testing.assert_close(pipe.images[b], imgs[b], rtol=0, atol=1e-6)
        torch.testing.assert_close(cap["dL"][b], dL[b], rtol=1e-4, atol=1e-6)
        torch.testing.assert_close(cap["grads"][b][0], g_means[b], rtol=1e-3, atol=1e-6)
    assert all(float(im.abs().sum()) > 0 for im in imgs)
