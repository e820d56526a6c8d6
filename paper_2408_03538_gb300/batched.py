"""Many scenes of uneven size and many lights through the whole path, one launch per stage.

The scenes are concatenated into one Gaussian set with CSR scene offsets. One BVH build covers
every scene (one radix tree with a subtree per scene), the transfer precompute is one packet
walk over the receivers of all scenes, the relight is one launch with each scene's own lights
(CUDA cores or the FP32-accurate BF16x3 split on the tensor cores, chosen by the autotuner),
and the render, the per-scene L2 losses, the render backward and the relight backward are
each one batched call over every scene (per-scene cameras of one image size). The whole step
is captured once into a CUDA graph and replayed, so a step costs one graph launch from the host.
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
        self.cams = list(cams)
        C = (order + 1) ** 2
        self.P = torch.empty((self.n, C), dtype=torch.float32, device=device)
        self.T = torch.empty((self.n, 3, C), dtype=torch.float32, device=device) if bounce else None
        self.idx = torch.empty((self.n, self.dirs.shape[0]), dtype=torch.int32, device=device) if bounce else None
        self.colors = torch.empty(3 * self.k * self.n, dtype=torch.float32, device=device)
        self.bg = torch.zeros(3, dtype=torch.float32, device=device)
        self.packet_dirs = 0
        self.walk = 0  # the autotuner may pick the per-ray walk (1)
        self.precision = L.PREC_FP32 if precision == "auto" else precision
        W, H = int(self.cams[0].width), int(self.cams[0].height)
        self.images = torch.empty((self.B, self.k, 3, H, W), dtype=torch.float32, device=device)
        self.state = None
        self._sizing_pass(device)
        if tune:
            bvh = api.build_bvh(self.g, self.offs_d)
            best = autotune.tune_transfer(self.g, bvh, self.dirs, order, bounce)
            self.walk, self.packet_dirs = (1, 0) if best == 0 else (0, best)
            if precision == "auto":
                Tt = self._transfer_out(bvh)
                self.precision = autotune.tune_relight_batched(Tt, self.g.albedo, self.offs_d, self.L, order)
        if targets is None:
            targets = torch.zeros_like(self.images)
        self.targets = torch.as_tensor(targets).to(device).reshape(self.images.shape).contiguous()
        self.graph = None
        self.frame_graph = None
        self.out = {}

    def scene(self, b) -> api.GaussianTensors:
        o0, o1 = int(self.offs_h[b]), int(self.offs_h[b + 1])
        g = self.g
        return api.GaussianTensors(g.means[o0:o1], g.scales[o0:o1], g.quats[o0:o1], g.opacity[o0:o1],
                                   g.normals[o0:o1], g.albedo[o0:o1])

    def _transfer_out(self, bvh):
        out = api.precompute_transfer(self.g, bvh, self.dirs, self.order, bounce=self.bounce,
                                      out={"P": self.P, "T": self.T, "idx": self.idx}, packet_dirs=self.packet_dirs,
                                      walk=self.walk)
        return out["T"] if self.bounce else self.P

    def _sizing_pass(self, device):
        """Capacity of the batched render state: the (Gaussian, tile) pairs of every scene."""
        bvh = api.build_bvh(self.g, self.offs_d)
        Tt = self._transfer_out(bvh)
        api.relight_batched(Tt, self.g.albedo, self.offs_d, self.L, self.order, L.PREC_FP32, out=self.colors)
        W, H = int(self.cams[0].width), int(self.cams[0].height)
        cap = max(16 * self.n, 1 << 16)
        while True:  # grow the probe until the pairs fit
            probe = api.RenderState(self.n, W, H, cap, device, n_scenes=self.B)
            st = api.Status(device)
            api.render_batched(self.g, self.offs_d, self.colors, self.k, self.cams, self.bg, probe, status=st,
                               out=self.images)
            torch.cuda.synchronize()
            if not (st.read() & L.STATUS_CAPACITY):
                break
            cap *= 4
        pairs = probe.n_pairs()
        del probe
        self.state = api.RenderState(self.n, W, H, int(pairs * 1.25) + 4096, device, n_scenes=self.B)

    def step(self, transfer: bool = True):
        """One pass of the whole path (forward and backward) over every scene: one call per stage.
        ``transfer=False`` runs the frame part only (relight, render, loss and both backward
        passes) on the transfer of the last full step: the geometry is frozen after the ray
        tracing (Sec. 4.4), so a training or serving loop repeats this part."""
        if transfer:
            bvh = api.build_bvh(self.g, self.offs_d)
            Tt = self._transfer_out(bvh)
        else:
            bvh = self.out.get("bvh")
            Tt = self.T if self.bounce else self.P
        api.relight_batched(Tt, self.g.albedo, self.offs_d, self.L, self.order, self.precision, out=self.colors)
        api.render_batched(self.g, self.offs_d, self.colors, self.k, self.cams, self.bg, self.state, out=self.images)
        losses, dimg = api.l2_loss_batched(self.images, self.targets)
        dm, ds, dq, do, dcol = api.render_backward_batched(self.g, self.offs_d, self.colors, self.k, self.cams,
                                                           self.bg, self.state, dimg)
        da, _, dL = api.relight_backward_batched(Tt, self.g.albedo, self.offs_d, self.L, self.order, dcol)
        self.out = {"losses": losses, "dL": dL, "grads": (dm, ds, dq, do, da), "bvh": bvh}
        return self.out

    def capture(self, transfer: bool = True):
        """Capture step(transfer) into a CUDA graph (after one eager warm-up on the capture stream);
        the full step and the frame part are kept as separate graphs."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.step(transfer)
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            captured = self.step(transfer)
        torch.cuda.synchronize()
        if transfer:
            self.graph, self.captured = graph, captured
        else:
            self.frame_graph, self.frame_captured = graph, captured
        return graph

    def replay(self, transfer: bool = True):
        if transfer:
            self.graph.replay()
            return self.captured
        self.frame_graph.replay()
        return self.frame_captured
