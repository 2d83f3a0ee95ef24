"""Serving-style batches: several frames of the same input rig rendered into
many target views of uneven size, as one CUDA graph.

Per frame f (in order, each refining against the previous frame):
    refine_depth -> weight_map            (one map per frame)
then ONE persistent launch fuses every (frame, target) item
    gvs_fuse_batch_launch                 (bundles pulled from a global counter)
and every (frame, target) pair is splatted with the fused depth as guide
    forward_splat.
The whole sequence is captured once into a torch.cuda.CUDAGraph and replayed
per batch; the fusion variant is chosen by the autotuner.
"""
from __future__ import annotations

import torch

from . import autotune, gvs


class BatchPlan:
    def __init__(self, in_cams, targets, rgba_frames, depth_frames, num_samples, z_near, z_far, mu, tau=0.03,
                 rgba_prev=None, state0=None, variant=None, graph=True):
        """rgba_frames / depth_frames: lists (one per frame) of device tensors int32 [N, H, W] /
        float32 [N, H, W].  rgba_prev / state0: the frame before the batch (None: the first frame
        takes its depth as is).  variant: fusion variant, or None to autotune."""
        self.cams, self.targets = list(in_cams), list(targets)
        self.F, self.N = len(rgba_frames), len(in_cams)
        self.rgba, self.depth = rgba_frames, depth_frames
        self.rgba_prev = rgba_prev
        self.cfg = dict(num_samples=num_samples, z_near=z_near, z_far=z_far, mu=mu, tau=tau)
        dev = depth_frames[0].device
        N, H, W = depth_frames[0].shape
        self.shape = (N, H, W)
        self.state0 = state0 if state0 is not None else depth_frames[0].clone()
        self.states = [torch.empty_like(depth_frames[0]) for _ in range(self.F)]
        self.masks = [torch.empty((N, H, W), dtype=torch.uint8, device=dev) for _ in range(self.F)]
        nb = gvs.fuse_workspace_bytes(N, W, H)
        self.maps = [gvs.workspace(nb, dev) for _ in range(self.F)]
        self.fused = [[torch.empty((t.height, t.width), dtype=torch.float32, device=dev) for t in self.targets]
                      for _ in range(self.F)]
        self.cross = [[torch.empty((t.height, t.width), dtype=torch.int16, device=dev) for t in self.targets]
                      for _ in range(self.F)]
        big = max(t.width * t.height for t in self.targets)
        # room for two z-buffers of the largest target (two views per splat pass; smaller
        # targets fit more), which stays L2-resident next to the streamed outputs
        self.ws_splat = gvs.workspace(2 * gvs.splat_workspace_bytes(N, big, 1), dev)
        self.splat = [[{k: torch.empty((N, t.height, t.width), dtype=dt, device=dev)
                        for k, dt in (("winner", torch.int32), ("warped_rgba", torch.int32),
                                      ("warped_depth", torch.float32), ("alpha", torch.uint8),
                                      ("guided", torch.uint8))} for t in self.targets] for _ in range(self.F)]
        self._prepare_maps()
        self.variant, self.timings = (variant, {}) if variant is not None else self._autotune()
        self.batch = self._make_batch(self.variant)
        self.graph = None
        if graph:
            self._capture()

    # -- pieces -------------------------------------------------------------------------------------
    def _refine_and_maps(self):
        c = self.cfg
        for f in range(self.F):
            prev_state = self.state0 if f == 0 else self.states[f - 1]
            self.states[f].copy_(prev_state)
            prev_rgba = self.rgba_prev if f == 0 else self.rgba[f - 1]
            gvs.refine_depth(self.rgba[f], prev_rgba, self.depth[f], self.states[f], self.masks[f], tau=c["tau"])
            gvs.weight_map(self.states[f], c["mu"], ws=self.maps[f])

    def _prepare_maps(self):
        self._refine_and_maps()
        torch.cuda.current_stream().synchronize()

    def _make_batch(self, variant):
        c = self.cfg
        items = [(self.maps[f], t, self.fused[f][n], self.cross[f][n])
                 for f in range(self.F) for n, t in enumerate(self.targets)]
        return gvs.FuseBatch(self.cams, items, c["num_samples"], c["z_near"], c["z_far"], c["mu"], variant=variant)

    def _autotune(self):
        c = self.cfg
        shape = {"views": self.shape, "targets": [(t.width, t.height) for t in self.targets], "frames": self.F,
                 "D": c["num_samples"], "z": (c["z_near"], c["z_far"]), "mu": c["mu"]}
        batches = {}

        def runner(v):
            batches[v] = self._make_batch(v)
            return batches[v].launch
        best, timings = autotune.choose(shape, runner, candidates=autotune.variants_for(len(self.cams)))
        for b in batches.values():
            b.close()
        return best, timings

    def _splats(self):
        for f in range(self.F):
            for n, t in enumerate(self.targets):
                gvs.forward_splat(self.cams, self.states[f], self.rgba[f], t, fused=self.fused[f][n],
                                  mu_guide=self.cfg["mu"], outputs=self.splat[f][n], ws=self.ws_splat)

    def _run_eager(self):
        self._refine_and_maps()
        self.batch.launch()
        self._splats()

    def _capture(self):
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            self._run_eager()  # warm up on the capture stream before recording
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._run_eager()
        torch.cuda.synchronize()

    # -- public -------------------------------------------------------------------------------------
    def run(self):
        """Enqueue the whole batch (graph replay when captured)."""
        if self.graph is not None:
            self.graph.replay()
        else:
            self._run_eager()

    def target_pixels(self) -> int:
        return self.F * sum(t.width * t.height for t in self.targets)

    def launches_per_run(self) -> int:
        n_refine = 1 + (1 if (self.N * self.shape[1] * self.shape[2]) % 4 else 0)
        per_frame = n_refine + 3                      # refine, weight map + two bound kernels
        per_splat = 0
        for t in self.targets:                        # key clear, scatter + resolve per group of views
            slots = max(1, min(self.N, self.ws_splat.numel() // (t.width * t.height * 8)))
            per_splat += 1 + 2 * ((self.N + slots - 1) // slots)
        return self.F * per_frame + 1 + self.F * per_splat
