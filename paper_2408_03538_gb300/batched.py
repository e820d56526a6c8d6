"""Many scenes of uneven size and many lights through the whole path in one replayable unit.

One BVH build covers every scene (one radix tree with a subtree per scene), the transfer
precompute is one persistent launch whose work counter runs over the receivers of all
scenes, and the relight is one launch with each scene's own lights (CUDA cores or tensor
cores, chosen by the autotuner). The per-scene splat renders, the L2 loss and the backward
passes follow on the same stream. The whole sequence is captured once into a CUDA graph
and replayed, so a step costs one graph launch from the host.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _lib as L
from . import api, autotune
from . import scenes as S


class BatchedPipeline:
    def __init__(self, scenes, dirs, order: int, lights, cams, targets=None, precision="auto", bounce=False,
                 device="cuda", tune=True):
        merged, offs = S.concat_scenes(scenes)
        self.B = len(scenes)
        self.order = order
        self.bounce = bounce
        self.offs_h = offs
        self.offs_d = torch.from_numpy(offs).to(device)
        self.g = api.GaussianTensors.from_scene(merged, device)
        self.n = self.g.n
        self.dirs = torch.from_numpy(np.ascontiguousarray(dirs)).to(device)
        self.L = torch.from_numpy(np.ascontiguousarray(lights, dtype=np.float32)).to(device)  # [B,k,3,C]
        self.k = int(self.L.shape[1])
        self.cams = cams
        C = (order + 1) ** 2
        self.P = torch.empty((self.n, C), dtype=torch.float32, device=device)
        self.T = torch.empty((self.n, 3, C), dtype=torch.float32, device=device) if bounce else None
        self.idx = torch.empty((self.n, self.dirs.shape[0]), dtype=torch.int32, device=device) if bounce else None
        self.colors = torch.empty(3 * self.k * self.n, dtype=torch.float32, device=device)
        self.bg = torch.zeros(3, dtype=torch.float32, device=device)
        self.index_buffer = 0
        self.precision = L.PREC_FP32 if precision == "auto" else precision
        # render states sized from one eager pass
        self.images = [torch.empty((self.k, 3, c.height, c.width), dtype=torch.float32, device=device)
                       for c in cams]
        self.states = [None] * self.B
        self._sizing_pass(device)
        if tune:
            bvh = api.build_bvh(self.g, self.offs_d)
            if bounce:
                self.index_buffer = autotune.tune_transfer(self.g, bvh, self.dirs, order, True)
            if precision == "auto" and not bounce:
                self.precision = autotune.tune_relight_batched(self.P, self.g.albedo, self.offs_d, self.L, order)
        if targets is None:
            targets = [torch.zeros_like(im) for im in self.images]
        self.targets = [t.to(device).contiguous() for t in targets]
        self.graph = None
        self.out = {}

    def scene(self, b) -> api.GaussianTensors:
        o0, o1 = int(self.offs_h[b]), int(self.offs_h[b + 1])
        g = self.g
        return api.GaussianTensors(g.means[o0:o1], g.scales[o0:o1], g.quats[o0:o1], g.opacity[o0:o1],
                                   g.normals[o0:o1], g.albedo[o0:o1])

    def _sizing_pass(self, device):
        bvh = api.build_bvh(self.g, self.offs_d)
        api.precompute_transfer(self.g, bvh, self.dirs, self.order, bounce=False, out={"P": self.P})
        api.relight_batched(self.P, self.g.albedo, self.offs_d, self.L, self.order, L.PREC_FP32, out=self.colors)
        for b in range(self.B):
            gb = self.scene(b)
            col = api.scene_colors(self.colors, self.k, self.offs_h, b)
            _, st = api.render(gb, col, self.cams[b], self.bg, max_pairs=max(64 * gb.n, 1 << 16))
            torch.cuda.synchronize()
            pairs = st.n_pairs()
            self.states[b] = api.RenderState(gb.n, self.cams[b].width, self.cams[b].height, int(pairs * 1.25) + 4096,
                                             device)

    def step(self):
        """One pass of the whole path (forward and backward) over every scene."""
        bvh = api.build_bvh(self.g, self.offs_d)
        out = api.precompute_transfer(self.g, bvh, self.dirs, self.order, bounce=self.bounce,
                                      out={"P": self.P, "T": self.T, "idx": self.idx},
                                      index_buffer=self.index_buffer)
        Tt = out["T"] if self.bounce else self.P
        prec = self.precision if not self.bounce else L.PREC_FP32
        api.relight_batched(Tt, self.g.albedo, self.offs_d, self.L, self.order, prec, out=self.colors)
        losses, dLs, grads = [], [], []
        for b in range(self.B):
            gb = self.scene(b)
            col = api.scene_colors(self.colors, self.k, self.offs_h, b)
            img, _ = api.render(gb, col, self.cams[b], self.bg, state=self.states[b], out=self.images[b])
            loss, dimg = api.l2_loss(img, self.targets[b])
            dm, ds, dq, do, dcol = api.render_backward(gb, col, self.cams[b], self.bg, self.states[b], dimg)
            o0, o1 = int(self.offs_h[b]), int(self.offs_h[b + 1])
            da, _, dL = api.relight_backward(Tt[o0:o1], gb.albedo, self.L[b], self.order, dcol)
            losses.append(loss)
            dLs.append(dL)
            grads.append((dm, ds, dq, do, da))
        self.out = {"losses": losses, "dL": dLs, "grads": grads, "bvh": bvh, "transfer": out}
        return self.out

    def capture(self):
        """Capture step() into a CUDA graph (after one eager warm-up on the capture stream)."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.step()
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.captured = self.step()
        torch.cuda.synchronize()
        return self.graph

    def replay(self):
        self.graph.replay()
        return self.captured
