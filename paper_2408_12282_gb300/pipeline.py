"""Device buffers, the per-step call sequence and the torch.autograd.Function.

One step (Fig. 2 of the paper, forward and backward) is the sequence
    mlp_fwd -> project_fwd -> bin_sort -> render_fwd            (forward)
    render_bwd -> mlp_bwd -> project_bwd                        (backward)
of C-ABI calls on one CUDA stream. PyTorch only owns the memory.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, replace

import numpy as np
import torch

from . import binding as B

SCENE_KEYS = ("mu", "log_s", "quat", "logit_o", "normal", "base", "rough", "metal", "sss", "vis")


def default_cfg(tile: int = 16) -> B.Cfg:
    c = B.cfg_default()
    c.tile = tile
    return c


class PairTable:
    """Host + device copies of a planned batch of view/light pairs."""

    def __init__(self, pairs, cfg: B.Cfg, scene_offsets=None, scene_counts=None, device="cuda"):
        n = len(pairs)
        self.h = (B.Pair * n)()
        for k, p in enumerate(pairs):
            q = self.h[k]
            R = np.asarray(p.R, np.float32).ravel()
            for i in range(9):
                q.R[i] = float(R[i])
            for i in range(3):
                q.t[i] = float(np.float32(p.t[i]))
                q.light[i] = float(np.float32(p.light[i]))
            q.fx, q.fy, q.cx, q.cy = float(p.fx), float(p.fy), float(p.cx), float(p.cy)
            q.W, q.H = int(p.W), int(p.H)
            s = getattr(p, "scene", 0)
            q.g_begin = int(scene_offsets[s]) if scene_offsets is not None else 0
            q.g_count = int(scene_counts[s]) if scene_counts is not None else 0
        self.info = B.plan(self.h, cfg)
        raw = np.frombuffer(bytes(self.h), dtype=np.uint8).copy()
        self.d = torch.from_numpy(raw).to(device)
        self.n = n

    @classmethod
    def from_structs(cls, h_pairs, cfg: B.Cfg, device="cuda"):
        """A table of copies of planned or unplanned pair structs (their
        caller-filled fields), planned with cfg."""
        t = cls.__new__(cls)
        n = len(h_pairs)
        t.h = (B.Pair * n)()
        for k in range(n):
            ctypes.memmove(ctypes.byref(t.h[k]), ctypes.byref(h_pairs[k]), ctypes.sizeof(B.Pair))
        t.info = B.plan(t.h, cfg)
        raw = np.frombuffer(bytes(t.h), dtype=np.uint8).copy()
        t.d = torch.from_numpy(raw).to(device)
        t.n = n
        return t

    @property
    def n_items(self):
        return int(self.info.n_items)

    @property
    def n_pixels(self):
        return int(self.info.n_pixels)

    @property
    def n_tiles(self):
        return int(self.info.n_tiles)


@dataclass
class MLPParams:
    kind: int
    precision: int
    W: list
    b: list

    def struct(self):
        return B.mlp_struct(self.kind, self.precision, self.W, self.b)


class GradientBuffers:
    """Every trainable-parameter gradient of a renderer in one flat float32
    buffer: the scene tensors (SCENE_KEYS order), the network's dW and db, and
    optional extra tensors (the SH visibility coefficients). Each is a
    contiguous view starting at a multiple of 64 floats (256 B). Zeroing is one
    fill, and the data-parallel exchange is one all-reduce of `flat`."""

    ALIGN = 64

    def __init__(self, scene_shapes: dict, w_shapes, b_shapes, extra_shapes=None, device="cuda"):
        specs = [("scene", k, tuple(v)) for k, v in scene_shapes.items()]
        specs += [("W", l, tuple(s)) for l, s in enumerate(w_shapes)]
        specs += [("b", l, tuple(s)) for l, s in enumerate(b_shapes)]
        specs += [("extra", k, tuple(v)) for k, v in (extra_shapes or {}).items()]
        offs, total = [], 0
        for _, _, shape in specs:
            offs.append(total)
            n = int(np.prod(shape)) if len(shape) else 1
            total += (n + self.ALIGN - 1) // self.ALIGN * self.ALIGN
        self.flat = torch.zeros(max(total, 1), device=device, dtype=torch.float32)
        self.scene, self.extra = {}, {}
        self.dW = [None] * len(w_shapes)
        self.db = [None] * len(b_shapes)
        for (kind, key, shape), o in zip(specs, offs):
            n = int(np.prod(shape)) if len(shape) else 1
            v = self.flat[o:o + n].view(shape)
            if kind == "scene":
                self.scene[key] = v
            elif kind == "W":
                self.dW[key] = v
            elif kind == "b":
                self.db[key] = v
            else:
                self.extra[key] = v

    def zero_(self):
        self.flat.zero_()


class _Group:
    """A run of consecutive pairs rendered with its own schedule (tile edge and
    per-block splat batch): its own pair table and tile lists. Its records,
    network rows, G-buffer, images and gradient records are slices of the
    renderer's buffers (a pair's items and pixels are contiguous)."""

    def __init__(self, r, p0: int, p1: int, cfg: B.Cfg):
        h = r.table.h
        self.cfg = cfg
        self.p0, self.p1 = p0, p1
        self.table = PairTable.from_structs(h[p0:p1], cfg, r.device)
        i0 = int(h[p0].item_offset)
        px0 = int(h[p0].pixel_offset)
        self.items = slice(i0, i0 + self.table.n_items)
        self.pixels = slice(px0, px0 + self.table.n_pixels)
        self.rec, self.rect, self.mlp_out = r.rec[self.items], r.rect[self.items], r.mlp_out[self.items]
        self.drec = r.drec[self.items]
        self.gbuf, self.last, self.img = r.gbuf[self.pixels], r.last[self.pixels], r.img[self.pixels]
        self.ranges = torch.zeros(self.table.n_tiles, 2, device=r.device, dtype=torch.int32)
        self.count = torch.zeros(1, device=r.device, dtype=torch.int64)
        self.stream = torch.cuda.Stream() if str(r.device).startswith("cuda") else None
        self.device = r.device
        self.capacity = 0

    def set_capacity(self, cap: int):
        self.capacity = int(cap)
        self.vals = torch.zeros(max(self.capacity, 1), device=self.device, dtype=torch.int32)
        wsb = B.bin_workspace_bytes(self.table.n_items, self.capacity, self.table.n_tiles)
        self.ws_bin = torch.empty(max(wsb, 256), device=self.device, dtype=torch.uint8)


class Renderer:
    """Owns every buffer of a batch and runs the forward/backward call sequence.

    schedule (optional): [(first pair, end pair, cfg), ...] covering the pairs
    in order. Each run of pairs is rendered with its own tile edge and
    per-block batch (cfg.tile, cfg.batch; e.g. one per scene from
    autotune_schedule): the projection, tile lists and render kernels run per
    run, each on its own stream inside the step (so one captured graph holds
    them all); the network and projection backward run once over all pairs."""

    def __init__(self, scene: dict, mlp: MLPParams, table: PairTable, cfg: B.Cfg, capacity: int | None = None,
                 fused: bool = True, device="cuda", vis_sh=None, shading: str = "deferred", schedule=None):
        """vis_sh (N x 16 device tensor, optional): the SH visibility term; v of
        each (pair, Gaussian) is then evaluated at the pair's light direction
        (sssgs_vis_sh_fwd) instead of read from scene["vis"].
        shading: "deferred" (Eq. 4 per pixel on the composited G-buffer, the
        paper's method) or "gaussian" (each Gaussian shaded at its mean and the
        colours composited: the paper's "w/o Deferred" ablation; unfused
        kernels, upstream gradient dimg or loss="paper")."""
        if shading not in ("deferred", "gaussian"):
            raise ValueError(f"unknown shading {shading!r}")
        self.shading = shading
        if shading == "gaussian":
            fused = False
        self.scene = scene
        self.mlp = mlp
        self.vis_sh = vis_sh
        self.table = table
        self.cfg = cfg
        self.fused = fused
        self.device = device
        n, P, T = table.n_items, table.n_pixels, table.n_tiles
        f32 = dict(device=device, dtype=torch.float32)
        i32 = dict(device=device, dtype=torch.int32)
        self.mlp_out = torch.zeros(n, 4, **f32)
        self.rec = torch.zeros(n, B.REC, **f32)
        self.rect = torch.zeros(n, 4, **i32)
        self.ranges = torch.zeros(T, 2, **i32)
        self.count = torch.zeros(1, device=device, dtype=torch.int64)
        self.status = torch.zeros(1, **i32)
        self.gbuf = torch.zeros(P, B.GBUF, **f32)
        self.last = torch.zeros(P, **i32)
        self.img = torch.zeros(P, 3, **f32)
        self.dgbuf = None if fused else torch.zeros(P, B.GBUF, **f32)
        self.rec_colors = torch.zeros(n, B.REC, **f32) if shading == "gaussian" else None
        self.drec = torch.zeros(n, B.REC, **f32)
        self.dx_items = torch.zeros(n, B.DX, **f32)
        self.grad_buffers = GradientBuffers({k: v.shape for k, v in scene.items()}, [w.shape for w in mlp.W],
                                            [b.shape for b in mlp.b],
                                            {"vis_sh": vis_sh.shape} if vis_sh is not None else None, device)
        self.grads = self.grad_buffers.scene
        self.dW = self.grad_buffers.dW
        self.db = self.grad_buffers.db
        self.vis_item = self.dvis_item = self.dvis_sh = None
        self.vis_traced = None
        self.loss_vis = None
        if vis_sh is not None:
            self.vis_item = torch.zeros(n, **f32)
            self.dvis_item = torch.zeros(n, **f32)
            self.dvis_sh = self.grad_buffers.extra["vis_sh"]
        self._scene_s = B.scene_struct(scene, self.vis_item)
        self._grad_s = B.scene_grad_struct(self.grads, self.dvis_item)
        self._mlp_s = mlp.struct()
        self._mlp_g = B.mlp_grad_struct(self.dW, self.db)
        mws = B.mlp_workspace_bytes(self._mlp_s, n)
        self.ws_mlp = torch.empty(max(mws, 256), device=device, dtype=torch.uint8)
        self.stats_fwd = None        # optional uint64[2] work counters (see sssgs_render_fwd/bwd)
        self.stats_bwd = None
        self.capacity = 0
        self.groups = None
        if schedule is not None and len(schedule) > 1:
            if vis_sh is not None or shading != "deferred" or not fused:
                raise ValueError("a per-run schedule takes the fused deferred path without the SH visibility term")
            ends = [(a, b) for a, b, _ in schedule]
            if ends[0][0] != 0 or ends[-1][1] != table.n or any(x[1] != y[0] for x, y in zip(ends, ends[1:])):
                raise ValueError("the schedule's runs must cover the pairs in order")
            self.groups = [_Group(self, a, b, c) for a, b, c in schedule]
            for g in self.groups:
                g.set_capacity(capacity if capacity is not None else max(1024, 16 * g.table.n_items))
        else:
            self.set_capacity(capacity if capacity is not None else max(1024, 16 * n))

    # ------------------------------------------------------------------ setup
    def set_capacity(self, cap: int):
        cap = int(cap)
        self.capacity = cap
        self.vals = torch.zeros(max(cap, 1), device=self.device, dtype=torch.int32)
        wsb = B.bin_workspace_bytes(self.table.n_items, cap, self.table.n_tiles)
        self.ws_bin = torch.empty(max(wsb, 256), device=self.device, dtype=torch.uint8)

    def fit_capacity(self, slack: float = 1.15):
        """Run the front end once and size the instance buffers (syncs).
        Returns the number of tile instances."""
        self.forward_front()
        torch.cuda.synchronize()
        if self.groups is not None:
            needs = [int(g.count.item()) for g in self.groups]
            if any(nd > g.capacity for nd, g in zip(needs, self.groups)) or self.status.item() != 0:
                for nd, g in zip(needs, self.groups):
                    if nd > g.capacity:
                        g.set_capacity(int(nd * slack) + 1024)
                self.status.zero_()
                self.forward_front()
                torch.cuda.synchronize()
            return sum(needs)
        need = int(self.count.item())
        if need > self.capacity or self.status.item() != 0:
            self.set_capacity(int(need * slack) + 1024)
            self.status.zero_()
            self.forward_front()
            torch.cuda.synchronize()
        return need

    # ------------------------------------------------------------------ runs of the schedule
    def _for_groups(self, fn, stream=None):
        """fn(group) for every run of the schedule, each on its own stream,
        forked from and joined back into the current (or given) stream."""
        cur = stream if stream is not None else torch.cuda.current_stream()
        for g in self.groups:
            g.stream.wait_stream(cur)
        for g in self.groups:
            with torch.cuda.stream(g.stream):
                fn(g)
        for g in self.groups:
            cur.wait_stream(g.stream)

    def _group_front(self, g):
        B.project_fwd(g.cfg, g.table.h, g.table.d, self._scene_s, g.mlp_out, g.rec, g.rect)
        B.bin_sort(g.cfg, g.table.h, g.table.d, g.rec, g.rect, g.capacity, g.vals, g.ranges, g.count,
                   self.status, g.ws_bin)

    def _group_render_fwd(self, g):
        B.render_fwd(g.cfg, g.table.h, g.table.d, g.rec, g.vals, g.ranges, g.gbuf, g.last, g.img, self.stats_fwd)

    def _group_render_bwd(self, g, dimg, target, weight, l1_scale):
        sl = g.pixels
        B.render_bwd(g.cfg, g.table.h, g.table.d, g.rec, g.vals, g.ranges, g.gbuf, g.last, g.img,
                     dimg[sl] if dimg is not None else None, target[sl] if target is not None else None,
                     weight[sl] if weight is not None else None, l1_scale, g.drec, self.stats_bwd)

    def run_stage(self, name, stream=None, dimg=None, target=None, weight=None, l1_scale=1.0):
        """One stage of the step over every pair (for per-stage timing):
        mlp_fwd, project_fwd, bin_sort, render_fwd, render_bwd (upstream dimg
        or the L1 loss against target), mlp_bwd, project_bwd."""
        t = self.table
        if name == "mlp_fwd":
            B.mlp_fwd(self._mlp_s, t.h, t.d, self._scene_s, self.mlp_out, self.status, stream)
        elif name == "mlp_bwd":
            B.mlp_bwd(self._mlp_s, t.h, t.d, self._scene_s, self.drec, self._mlp_g, self.dx_items, self.ws_mlp,
                      self.status, stream)
        elif name == "project_bwd":
            B.project_bwd(self.cfg, t.h, t.d, self._scene_s, self.drec, self.dx_items, self._grad_s, stream)
        elif self.groups is not None:
            fn = {"project_fwd": lambda g: B.project_fwd(g.cfg, g.table.h, g.table.d, self._scene_s, g.mlp_out,
                                                         g.rec, g.rect),
                  "bin_sort": lambda g: B.bin_sort(g.cfg, g.table.h, g.table.d, g.rec, g.rect, g.capacity, g.vals,
                                                   g.ranges, g.count, self.status, g.ws_bin),
                  "render_fwd": self._group_render_fwd,
                  "render_bwd": lambda g: self._group_render_bwd(g, dimg, target, weight, l1_scale)}[name]
            self._for_groups(fn, stream)
        elif name == "project_fwd":
            B.project_fwd(self.cfg, t.h, t.d, self._scene_s, self.mlp_out, self.rec, self.rect, stream)
        elif name == "bin_sort":
            B.bin_sort(self.cfg, t.h, t.d, self.rec, self.rect, self.capacity, self.vals, self.ranges, self.count,
                       self.status, self.ws_bin, stream)
        elif name == "render_fwd":
            B.render_fwd(self.cfg, t.h, t.d, self.rec, self.vals, self.ranges, self.gbuf, self.last, self.img,
                         self.stats_fwd, stream)
        elif name == "render_bwd":
            B.render_bwd(self.cfg, t.h, t.d, self.rec, self.vals, self.ranges, self.gbuf, self.last, self.img,
                         dimg, target, weight, l1_scale, self.drec, self.stats_bwd, stream)
        else:
            raise ValueError(f"unknown stage {name!r}")

    # ------------------------------------------------------------------ steps
    def forward_front(self, stream=None, render=False):
        t = self.table
        if self.groups is not None:
            B.mlp_fwd(self._mlp_s, t.h, t.d, self._scene_s, self.mlp_out, self.status, stream)

            def front(g):
                self._group_front(g)
                if render:
                    self._group_render_fwd(g)
            self._for_groups(front, stream)
            return
        if self.vis_sh is not None:
            B.vis_sh_fwd(t.h, t.d, self._scene_s, self.vis_sh, self.vis_item, stream)
        B.mlp_fwd(self._mlp_s, t.h, t.d, self._scene_s, self.mlp_out, self.status, stream)
        B.project_fwd(self.cfg, t.h, t.d, self._scene_s, self.mlp_out, self.rec, self.rect, stream)
        B.bin_sort(self.cfg, t.h, t.d, self.rec, self.rect, self.capacity, self.vals, self.ranges, self.count,
                   self.status, self.ws_bin, stream)

    def forward(self, stream=None):
        if self.groups is not None:
            self.forward_front(stream, render=True)
            return self.img
        self.forward_front(stream)
        t = self.table
        if self.shading == "gaussian":
            B.shade_gaussians_fwd(t.h, t.d, self._scene_s, self.rec, self.rec_colors, stream)
            B.composite_fwd(self.cfg, t.h, t.d, self.rec_colors, self.vals, self.ranges, self.gbuf, self.last,
                            stream)
            B.colors_to_image(t.h, self.gbuf, self.img, stream)
        elif self.fused:
            B.render_fwd(self.cfg, t.h, t.d, self.rec, self.vals, self.ranges, self.gbuf, self.last, self.img,
                         self.stats_fwd, stream)
        else:
            B.composite_fwd(self.cfg, t.h, t.d, self.rec, self.vals, self.ranges, self.gbuf, self.last, stream)
            B.shade_fwd(self.cfg, t.h, t.d, self.gbuf, self.img, stream)
        return self.img

    def zero_grads(self):
        self.drec.zero_()
        self.grad_buffers.zero_()
        if self.vis_sh is not None:
            self.dvis_item.zero_()

    def exchange_gradients(self, group=None):
        """Data-parallel exchange: sum every parameter gradient over the
        process group with one all-reduce of the flat gradient buffer."""
        exchange_gradients(self.grad_buffers.flat, group)

    def trace_visibility(self, stream=None):
        """Ray-traced visibility of every (pair, Gaussian) toward the pair's
        light (BVH over the current geometry) into self.vis_traced: the target
        of the ray-traced visibility loss."""
        n = self.scene["mu"].shape[0]
        if getattr(self, "bvh", None) is None:
            self.bvh = torch.empty(B.bvh_floats(n), device=self.device, dtype=torch.float32)
            self.ws_bvh = torch.empty(B.bvh_workspace_bytes(n), device=self.device, dtype=torch.uint8)
            self.vis_traced = torch.zeros(self.table.n_items, device=self.device, dtype=torch.float32)
        B.bvh_build(self.cfg, self._scene_s, self.bvh, self.ws_bvh, stream)
        B.trace_visibility(self.cfg, self.table.h, self.table.d, self._scene_s, self.bvh, self.vis_traced, stream)
        return self.vis_traced

    def _loss_buffers(self):
        if getattr(self, "loss", None) is None:
            n, P = self.table.n_items, self.table.n_pixels
            self.loss = torch.zeros(self.table.n, device=self.device, dtype=torch.float32)
            self.dimg_loss = torch.zeros(P, 3, device=self.device, dtype=torch.float32)
            self.ws_loss = torch.empty(B.image_loss_workspace_bytes(P), device=self.device, dtype=torch.uint8)

    def backward(self, dimg=None, target=None, weight=None, l1_scale=1.0, stream=None, loss="l1",
                 lambda_dssim=0.2, lambda_incident=0.02, lambda_raytrace=0.01):
        """Backward of one step. loss="l1": the upstream gradient is dimg, or
        (dimg None) the fused L1 loss against target. loss="paper": the training
        losses of App. E: image loss (1 - lambda_dssim) L1 + lambda_dssim
        (1 - SSIM) against target plus the incident-light constraint; the
        per-pair loss values land in self.loss. With the SH visibility term
        and a traced target (trace_visibility), the ray-traced visibility loss
        (weight lambda_raytrace) is added and its per-pair values land in
        self.loss_vis."""
        t = self.table
        self.zero_grads()
        if loss == "paper":
            if target is None:
                raise ValueError("the paper's losses take a target")
            self._loss_buffers()
            self.loss.zero_()
            B.image_loss(self.cfg, t.h, t.d, self.img, target, lambda_dssim, self.dimg_loss, self.loss,
                         self.ws_loss, stream)
            if self.shading == "gaussian":
                self._backward_gaussian_shading(self.dimg_loss, stream)
            elif self.groups is not None:
                self._for_groups(lambda g: self._group_render_bwd(g, self.dimg_loss, None, None, 1.0), stream)
            elif self.fused:
                B.render_bwd(self.cfg, t.h, t.d, self.rec, self.vals, self.ranges, self.gbuf, self.last, self.img,
                             self.dimg_loss, None, None, 1.0, self.drec, self.stats_bwd, stream)
            else:
                raise ValueError("the paper's losses run on the fused path")
            B.incident_loss(t.h, t.d, self.rec, lambda_incident, self.drec, self.loss, stream)
        elif loss != "l1":
            raise ValueError(f"unknown loss {loss!r}")
        elif self.shading == "gaussian":
            if dimg is None:
                raise ValueError("per-Gaussian shading takes dimg (or loss='paper')")
            self._backward_gaussian_shading(dimg, stream)
        elif self.groups is not None:
            self._for_groups(lambda g: self._group_render_bwd(g, dimg, target, weight, l1_scale), stream)
        elif self.fused:
            B.render_bwd(self.cfg, t.h, t.d, self.rec, self.vals, self.ranges, self.gbuf, self.last, self.img,
                         dimg, target, weight, l1_scale, self.drec, self.stats_bwd, stream)
        else:
            if dimg is None:
                raise ValueError("the unfused path takes dimg")
            B.shade_bwd(self.cfg, t.h, t.d, self.gbuf, dimg, self.dgbuf, stream)
            B.composite_bwd(self.cfg, t.h, t.d, self.rec, self.vals, self.ranges, self.gbuf, self.last, self.dgbuf,
                            self.drec, stream)
        B.mlp_bwd(self._mlp_s, t.h, t.d, self._scene_s, self.drec, self._mlp_g, self.dx_items, self.ws_mlp,
                  self.status, stream)
        B.project_bwd(self.cfg, t.h, t.d, self._scene_s, self.drec, self.dx_items, self._grad_s, stream)
        if self.vis_sh is not None:
            if self.vis_traced is not None and lambda_raytrace > 0.0:
                if self.loss_vis is None:
                    self.loss_vis = torch.zeros(t.n, device=self.device, dtype=torch.float32)
                self.loss_vis.zero_()
                B.vis_loss(t.h, t.d, self.vis_item, self.vis_traced, lambda_raytrace, self.dvis_item, self.loss_vis,
                           stream)
            B.vis_sh_bwd(t.h, t.d, self._scene_s, self.vis_sh, self.dvis_item, self.dvis_sh, self.grads["mu"],
                         stream)

    def _backward_gaussian_shading(self, dimg, stream):
        t = self.table
        B.colors_to_image_bwd(t.h, dimg, self.dgbuf, stream)
        B.composite_bwd(self.cfg, t.h, t.d, self.rec_colors, self.vals, self.ranges, self.gbuf, self.last,
                        self.dgbuf, self.drec, stream)
        B.shade_gaussians_bwd(t.h, t.d, self._scene_s, self.rec, self.drec, stream)

    def capture(self, dimg=None, target=None, weight=None, l1_scale=1.0, loss="l1"):
        """Capture one forward + backward step as a CUDA graph and return it.

        The step has no host synchronisation (instance buffers are sized by
        capacity, counts stay on the device), so it can be replayed as is;
        call fit_capacity() first. Inputs are read from the same buffers at
        every replay."""
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            self.forward()
            self.backward(dimg=dimg, target=target, weight=weight, l1_scale=l1_scale, loss=loss)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, capture_error_mode="thread_local"):
            self.forward()
            self.backward(dimg=dimg, target=target, weight=weight, l1_scale=l1_scale, loss=loss)
        torch.cuda.synchronize()
        return g

    def check_status(self):
        s = int(self.status.item())
        if s & B.STATUS_CAPACITY:
            if self.groups is not None:
                need = [(g.capacity, int(g.count.item())) for g in self.groups]
                raise B.SSSGSError(f"instance capacity exceeded in a run of the schedule (capacity, needed): {need}")
            raise B.SSSGSError(f"instance capacity {self.capacity} exceeded ({int(self.count.item())} needed)")
        if s & B.STATUS_TIMEOUT:
            raise B.SSSGSError("a tensor-core kernel stopped on its wait limit; outputs are incomplete")

    @property
    def n_instances(self) -> int:
        """Tile instances of the last binning (syncs)."""
        if self.groups is not None:
            return sum(int(g.count.item()) for g in self.groups)
        return int(self.count.item())


class SSSRenderFunction(torch.autograd.Function):
    """Differentiable OLAT render: (scene params, MLP weights) -> image (pixels x 3)."""

    @staticmethod
    def forward(ctx, renderer: Renderer, *params):
        renderer.forward()
        ctx.renderer = renderer
        return renderer.img.clone()

    @staticmethod
    def backward(ctx, dimg):
        r = ctx.renderer
        r.backward(dimg=dimg.contiguous())
        return (None, *[r.grads[k] for k in SCENE_KEYS], *r.dW, *r.db)


def render(renderer: Renderer):
    params = [renderer.scene[k] for k in SCENE_KEYS] + list(renderer.mlp.W) + list(renderer.mlp.b)
    return SSSRenderFunction.apply(renderer, *params)


# ---------------------------------------------------------------------- helpers

def scene_to_device(scene, device="cuda") -> dict:
    """scenegen.Scene -> dict of contiguous float32 device tensors."""
    out = {}
    for k in SCENE_KEYS:
        a = np.ascontiguousarray(getattr(scene, k), dtype=np.float32)
        out[k] = torch.from_numpy(a).to(device).requires_grad_(False)
    return out


def concat_scenes(scenes, device="cuda"):
    """Concatenate several scenegen.Scene objects; returns (dict, offsets, counts)."""
    offs, counts, acc = [], [], 0
    for s in scenes:
        offs.append(acc)
        counts.append(s.N)
        acc += s.N
    out = {}
    for k in SCENE_KEYS:
        a = np.concatenate([np.asarray(getattr(s, k), np.float32) for s in scenes], axis=0)
        out[k] = torch.from_numpy(np.ascontiguousarray(a)).to(device)
    return out, offs, counts


def mlp_to_device(spec, precision=None, device="cuda") -> MLPParams:
    kind = {"basic": B.MLP_BASIC, "pe6": B.MLP_PE6, "paper": B.MLP_PAPER}[spec.kind]
    prec = precision if precision is not None else (B.BF16 if spec.precision == "bf16" else B.FP32)
    W = [torch.from_numpy(np.ascontiguousarray(w, np.float32)).to(device) for w in spec.weights]
    b = [torch.from_numpy(np.ascontiguousarray(x, np.float32)).to(device) for x in spec.biases]
    return MLPParams(kind, prec, W, b)


def renderer_for_workload(wl, precision=None, fused=True, tile=None, capacity=None, device="cuda",
                          pair_slice=None, vis_sh=None, shading="deferred", batch=None,
                          scene_cfgs=None) -> Renderer:
    """vis_sh: optional N x 16 numpy array of SH visibility coefficients.
    tile, batch: the schedule of every pair. scene_cfgs: one B.Cfg per scene
    (autotune_schedule), each run of consecutive pairs of a scene rendered
    with its scene's tile edge and batch."""
    cfg = default_cfg(tile or wl.tile)
    if batch is not None:
        cfg.batch = int(batch)
    scene, offs, counts = concat_scenes(wl.scenes, device)
    pairs = wl.pairs if pair_slice is None else wl.pairs[pair_slice]
    schedule = None
    if scene_cfgs is not None:
        runs = []
        for k, p in enumerate(pairs):
            if runs and runs[-1][2] == p.scene:
                runs[-1][1] = k + 1
            else:
                runs.append([k, k + 1, p.scene])
        schedule = [(a, b, scene_cfgs[sc]) for a, b, sc in runs]
        keys = {(c.tile, c.batch) for _, _, c in schedule}
        if len(keys) == 1:          # one schedule for all: the plain single-run path
            cfg = schedule[0][2]
            schedule = None
    table = PairTable(pairs, cfg, offs, counts, device)
    mlp = mlp_to_device(wl.mlp, precision, device)
    sh = None
    if vis_sh is not None:
        sh = torch.from_numpy(np.ascontiguousarray(vis_sh, np.float32)).to(device)
    return Renderer(scene, mlp, table, cfg, capacity=capacity, fused=fused, device=device, vis_sh=sh,
                    shading=shading, schedule=schedule)


class MultiLightRenderer:
    """A batch of views, each under the same number of point lights: the
    light-stage batches of the paper's OLAT data (Sec. 4.1), or a relit view as
    a weighted sum of OLAT renders (App. C "Image Based Lighting").

    Projection, binning/sort and the compositing alphas run once per view
    (table `views`); the network runs per (view, light) pair (table `pairs`,
    view-major), and the render kernels composite the light channels and shade
    every light of a view in one pass. Images come out per (view, light) pair
    in pair order, or per view as a weighted sum (forward(env_w=...))."""

    def __init__(self, scene: dict, mlp: MLPParams, views, lights, cfg: B.Cfg, scene_offsets, scene_counts,
                 capacity: int | None = None, device="cuda", vis_sh=None):
        """vis_sh (N x 16 device tensor, optional): the SH visibility term,
        evaluated per (view, light) pair at the light direction; v enters the
        network per pair (the composited visibility channel does not enter the
        shading, so the per-view records keep the per-Gaussian v)."""
        lights = np.asarray(lights, np.float64)
        V, L = lights.shape[0], lights.shape[1]
        if len(views) != V or lights.shape[2] != 3:
            raise ValueError("lights must be n_views x n_lights x 3")
        self.scene, self.mlp, self.cfg, self.device, self.n_lights = scene, mlp, cfg, device, L
        self.views = PairTable(views, cfg, scene_offsets, scene_counts, device)
        pairs = [replace(v, light=lights[k][l]) for k, v in enumerate(views) for l in range(L)]
        self.pairs = PairTable(pairs, cfg, scene_offsets, scene_counts, device)
        self.lights = torch.from_numpy(np.ascontiguousarray(lights.reshape(-1), np.float32)).to(device)
        nv, npi, Pv, Pp, T = (self.views.n_items, self.pairs.n_items, self.views.n_pixels, self.pairs.n_pixels,
                              self.views.n_tiles)
        f32 = dict(device=device, dtype=torch.float32)
        i32 = dict(device=device, dtype=torch.int32)
        self.mlp_out = torch.zeros(npi, 4, **f32)
        self.rec = torch.zeros(nv, B.REC, **f32)
        self.rect = torch.zeros(nv, 4, **i32)
        self.ranges = torch.zeros(T, 2, **i32)
        self.count = torch.zeros(1, device=device, dtype=torch.int64)
        self.status = torch.zeros(1, **i32)
        self.gbuf = torch.zeros(Pv, 12 + 4 * L, **f32)
        self.last = torch.zeros(Pv, **i32)
        self.img = torch.zeros(Pp, 3, **f32)
        self.drec = torch.zeros(nv, B.REC, **f32)
        self.dmlp = torch.zeros(npi, 4, **f32)
        self.dx_items = torch.zeros(npi, B.DX, **f32)
        self.grad_buffers = GradientBuffers({k: v.shape for k, v in scene.items()}, [w.shape for w in mlp.W],
                                            [b.shape for b in mlp.b],
                                            {"vis_sh": vis_sh.shape} if vis_sh is not None else None, device)
        self.grads = self.grad_buffers.scene
        self.dW = self.grad_buffers.dW
        self.db = self.grad_buffers.db
        self.vis_sh = vis_sh
        self.vis_item = self.dvis_item = self.dvis_sh = self.vis_traced = self.loss_vis = None
        if vis_sh is not None:
            self.vis_item = torch.zeros(npi, **f32)
            self.dvis_item = torch.zeros(npi, **f32)
            self.dvis_sh = self.grad_buffers.extra["vis_sh"]
        self._scene_s = B.scene_struct(scene)                       # per-view records
        self._grad_s = B.scene_grad_struct(self.grads)
        self._scene_p = B.scene_struct(scene, self.vis_item)        # (view, light) pairs: network
        self._grad_p = B.scene_grad_struct(self.grads, self.dvis_item)
        self._mlp_s = mlp.struct()
        self._mlp_g = B.mlp_grad_struct(self.dW, self.db)
        mws = B.mlp_workspace_bytes(self._mlp_s, npi)
        self.ws_mlp = torch.empty(max(mws, 256), device=device, dtype=torch.uint8)
        self.stats_fwd = None
        self.stats_bwd = None
        self.capacity = 0
        self.set_capacity(capacity if capacity is not None else max(1024, 16 * nv))

    def set_capacity(self, cap: int):
        self.capacity = int(cap)
        self.vals = torch.zeros(max(self.capacity, 1), device=self.device, dtype=torch.int32)
        wsb = B.bin_workspace_bytes(self.views.n_items, self.capacity, self.views.n_tiles)
        self.ws_bin = torch.empty(max(wsb, 256), device=self.device, dtype=torch.uint8)

    def fit_capacity(self, slack: float = 1.15):
        self.forward_front()
        torch.cuda.synchronize()
        need = int(self.count.item())
        if need > self.capacity or self.status.item() != 0:
            self.set_capacity(int(need * slack) + 1024)
            self.status.zero_()
            self.forward_front()
            torch.cuda.synchronize()
        return need

    def forward_front(self, stream=None):
        v, p = self.views, self.pairs
        if self.vis_sh is not None:
            B.vis_sh_fwd(p.h, p.d, self._scene_p, self.vis_sh, self.vis_item, stream)
        B.mlp_fwd(self._mlp_s, p.h, p.d, self._scene_p, self.mlp_out, self.status, stream)
        B.project_fwd(self.cfg, v.h, v.d, self._scene_s, None, self.rec, self.rect, stream)
        B.bin_sort(self.cfg, v.h, v.d, self.rec, self.rect, self.capacity, self.vals, self.ranges, self.count,
                   self.status, self.ws_bin, stream)

    def forward(self, stream=None, env_w=None, out=None):
        """Per-(view, light) images into self.img; with env_w (device
        float[n_views * n_lights]) the weighted sum per view into `out`
        (n_view_pixels x 3)."""
        if env_w is not None and out is None:
            raise ValueError("forward(env_w=...) writes the weighted image into `out`; pass it")
        self.forward_front(stream)
        v = self.views
        img = self.img if env_w is None else out
        B.render_ml_fwd(self.cfg, v.h, v.d, self.n_lights, self.lights, self.rec, self.mlp_out, self.vals,
                        self.ranges, self.gbuf, self.last, img, env_w, self.stats_fwd, stream)
        self._pair_images_current = env_w is None
        return img

    def zero_grads(self):
        self.drec.zero_()
        self.dmlp.zero_()
        self.grad_buffers.zero_()
        if self.vis_sh is not None:
            self.dvis_item.zero_()

    def exchange_gradients(self, group=None):
        """One all-reduce of the flat gradient buffer (see Renderer)."""
        exchange_gradients(self.grad_buffers.flat, group)

    def trace_visibility(self, stream=None):
        """Ray-traced visibility of every (view, light, Gaussian) toward its
        light into self.vis_traced (the target of the visibility loss)."""
        n = self.scene["mu"].shape[0]
        if getattr(self, "bvh", None) is None:
            self.bvh = torch.empty(B.bvh_floats(n), device=self.device, dtype=torch.float32)
            self.ws_bvh = torch.empty(B.bvh_workspace_bytes(n), device=self.device, dtype=torch.uint8)
            self.vis_traced = torch.zeros(self.pairs.n_items, device=self.device, dtype=torch.float32)
        B.bvh_build(self.cfg, self._scene_s, self.bvh, self.ws_bvh, stream)
        B.trace_visibility(self.cfg, self.pairs.h, self.pairs.d, self._scene_s, self.bvh, self.vis_traced, stream)
        return self.vis_traced

    def backward(self, dimg=None, target=None, l1_scale=1.0, stream=None, lambda_raytrace=0.01):
        """Upstream: dimg per (view, light) image, or the L1 loss against target
        (which reads the per-(view, light) images of the last forward)."""
        if dimg is None and not getattr(self, "_pair_images_current", False):
            raise ValueError("the L1 upstream needs the per-(view, light) images: run forward() without "
                             "env_w before backward(target=...), or pass dimg")
        v, p = self.views, self.pairs
        self.zero_grads()
        B.render_ml_bwd(self.cfg, v.h, v.d, self.n_lights, self.lights, self.rec, self.mlp_out, self.vals,
                        self.ranges, self.gbuf, self.last, self.img, dimg, target, l1_scale, self.drec, self.dmlp,
                        self.stats_bwd, stream)
        B.mlp_bwd_strided(self._mlp_s, p.h, p.d, self._scene_p, self.dmlp, 4, self._mlp_g, self.dx_items,
                          self.ws_mlp, self.status, stream)
        B.project_bwd(self.cfg, v.h, v.d, self._scene_s, self.drec, None, self._grad_s, stream)
        B.project_bwd(self.cfg, p.h, p.d, self._scene_p, None, self.dx_items, self._grad_p, stream)
        if self.vis_sh is not None:
            if self.vis_traced is not None and lambda_raytrace > 0.0:
                if self.loss_vis is None:
                    self.loss_vis = torch.zeros(p.n, device=self.device, dtype=torch.float32)
                self.loss_vis.zero_()
                B.vis_loss(p.h, p.d, self.vis_item, self.vis_traced, lambda_raytrace, self.dvis_item,
                           self.loss_vis, stream)
            B.vis_sh_bwd(p.h, p.d, self._scene_p, self.vis_sh, self.dvis_item, self.dvis_sh, self.grads["mu"],
                         stream)

    def capture(self, dimg=None, target=None, l1_scale=1.0):
        """One forward + backward step as a CUDA graph (call fit_capacity() first)."""
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            self.forward()
            self.backward(dimg=dimg, target=target, l1_scale=l1_scale)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, capture_error_mode="thread_local"):
            self.forward()
            self.backward(dimg=dimg, target=target, l1_scale=l1_scale)
        torch.cuda.synchronize()
        return g

    def check_status(self):
        s = int(self.status.item())
        if s & B.STATUS_CAPACITY:
            raise B.SSSGSError(f"instance capacity {self.capacity} exceeded ({int(self.count.item())} needed)")
        if s & B.STATUS_TIMEOUT:
            raise B.SSSGSError("a tensor-core kernel stopped on its wait limit; outputs are incomplete")


def multilight_renderer_for_workload(wl, precision=None, capacity=None, device="cuda",
                                     vis_sh=None) -> MultiLightRenderer:
    """Views and lights of a workload whose pairs come in runs of wl.n_lights
    sharing a camera (scenegen c6)."""
    L = wl.n_lights
    if len(wl.pairs) % L:
        raise ValueError("pair count is not a multiple of n_lights")
    views = wl.pairs[::L]
    lights = np.array([[p.light for p in wl.pairs[k:k + L]] for k in range(0, len(wl.pairs), L)])
    cfg = default_cfg(16)
    scene, offs, counts = concat_scenes(wl.scenes, device)
    mlp = mlp_to_device(wl.mlp, precision, device)
    sh = None
    if vis_sh is not None:
        sh = torch.from_numpy(np.ascontiguousarray(vis_sh, np.float32)).to(device)
    return MultiLightRenderer(scene, mlp, views, lights, cfg, offs, counts, capacity=capacity, device=device,
                              vis_sh=sh)


def autotune_schedule(wl, precision=None, tiles=(8, 16, 32), batches=(32, 64), reps=3, device="cuda",
                      slack: float = 1.1, instances_per_item: float = 16.0):
    """Pick the tile edge and per-block splat batch of every scene of a
    workload by measurement (sssgs_autotune): for each scene, its pairs'
    schedule-dependent stages (projection, binning + sort, fused render
    forward and backward) are timed on the device for every candidate.
    Returns (one B.Cfg per scene, {scene: [TuneResult, ...]}). Blocking.
    The first trial sizes the instance buffers at instances_per_item per
    (pair, Gaussian); candidates that need more are rerun with buffers sized
    from their reported counts."""
    base = default_cfg(16)
    r = renderer_for_workload(wl, precision=precision, device=device)
    r.run_stage("mlp_fwd")
    torch.cuda.synchronize()
    h = r.table.h
    cfgs, table = [], {}
    for sc in range(len(wl.scenes)):
        ks = [k for k, p in enumerate(wl.pairs) if p.scene == sc]
        sub = PairTable.from_structs([h[k] for k in ks], base, device)
        rows = [r.mlp_out[int(h[k].item_offset):int(h[k].item_offset) + int(h[k].g_count)] for k in ks]
        mlp_out = torch.cat(rows).contiguous()
        n, P = sub.n_items, sub.n_pixels
        max_tiles = PairTable.from_structs(sub.h, default_cfg(min(tiles)), device).n_tiles
        f32 = dict(device=device, dtype=torch.float32)
        keep = dict(d_pairs=torch.zeros(sub.n * ctypes.sizeof(B.Pair), device=device, dtype=torch.uint8),
                    rec=torch.zeros(n, B.REC, **f32), rect=torch.zeros(n, 4, device=device, dtype=torch.int32),
                    ranges=torch.zeros(max_tiles, 2, device=device, dtype=torch.int32),
                    count=torch.zeros(1, device=device, dtype=torch.int64),
                    status=torch.zeros(1, device=device, dtype=torch.int32),
                    gbuf=torch.zeros(P, B.GBUF, **f32), last=torch.zeros(P, device=device, dtype=torch.int32),
                    img=torch.zeros(P, 3, **f32), drec=torch.zeros(n, B.REC, **f32),
                    dimg=torch.full((P, 3), 1e-6, **f32))

        def buffers(capacity):
            keep["vals"] = torch.zeros(max(capacity, 1), device=device, dtype=torch.int32)
            keep["ws"] = torch.empty(max(B.bin_workspace_bytes(n, capacity, max_tiles), 256), device=device,
                                     dtype=torch.uint8)
            tb = B.TuneBuffers()
            for k in ("d_pairs", "rec", "rect", "vals", "ranges", "gbuf", "last", "img", "drec", "dimg"):
                setattr(tb, k, keep[k].data_ptr())
            tb.capacity, tb.max_tiles = int(capacity), int(max_tiles)
            tb.d_count, tb.d_status = keep["count"].data_ptr(), keep["status"].data_ptr()
            tb.workspace, tb.workspace_bytes = keep["ws"].data_ptr(), keep["ws"].numel()
            return tb

        capacity = int(instances_per_item * n) + 1024
        best, res = B.autotune(base, sub.h, r._scene_s, mlp_out, buffers(capacity), tiles, batches, reps)
        short = [x for x in res if x.status == B.STATUS_CAPACITY]
        if short:                       # rerun the candidates whose instances did not fit (counts reported)
            capacity = int(max(x.instances for x in short) * slack) + 1024
            retry_tiles = sorted({x.tile for x in short})
            _, res2 = B.autotune(base, sub.h, r._scene_s, mlp_out, buffers(capacity), retry_tiles, batches, reps)
            got = {(x.tile, x.batch): x for x in res2}
            res = [got.get((x.tile, x.batch), x) for x in res]
            ok = [x for x in res if x.status == 0]
            fastest = min(ok, key=lambda x: x.ms)
            best = default_cfg(fastest.tile)
            best.batch = fastest.batch
        cfgs.append(best)
        table[sc] = res
        del keep
        torch.cuda.empty_cache()
    del r
    torch.cuda.empty_cache()
    return cfgs, table


# ---------------------------------------------------------------------- data parallel

def shard_pairs(n_pairs: int, rank: int, world: int) -> list:
    """Pairs owned by `rank` when a batch of view/light pairs is split over
    `world` processes (round-robin, so uneven batches stay balanced)."""
    return list(range(rank, n_pairs, world))


def exchange_gradients(flat, group=None):
    """Sum the flat gradient buffer (GradientBuffers.flat) over the process
    group with one all-reduce: the one exchange of a data-parallel step
    (renders of different pairs are independent; the parameters are shared)."""
    import torch.distributed as dist
    dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)


# ---------------------------------------------------------------------- checkpoint / resume

CHECKPOINT_FORMAT = "sssgs-checkpoint-1"


def state_dict(renderer) -> dict:
    """The trainable state of a Renderer or MultiLightRenderer as CPU tensors:
    scene parameters, network weights and biases, and the SH visibility
    coefficients when the renderer has them."""
    sd = {f"scene.{k}": renderer.scene[k].detach().cpu().clone() for k in SCENE_KEYS}
    for l, w in enumerate(renderer.mlp.W):
        sd[f"mlp.W{l}"] = w.detach().cpu().clone()
    for l, b in enumerate(renderer.mlp.b):
        sd[f"mlp.b{l}"] = b.detach().cpu().clone()
    if getattr(renderer, "vis_sh", None) is not None:
        sd["vis_sh"] = renderer.vis_sh.detach().cpu().clone()
    return sd


def load_state_dict(renderer, sd: dict) -> None:
    """Copy a state_dict into the renderer's existing buffers, in place, so a
    captured CUDA graph keeps reading the restored values. Raises ValueError
    on a missing, unexpected or mis-shaped entry (nothing is copied then)."""
    targets = {f"scene.{k}": renderer.scene[k] for k in SCENE_KEYS}
    targets.update({f"mlp.W{l}": w for l, w in enumerate(renderer.mlp.W)})
    targets.update({f"mlp.b{l}": b for l, b in enumerate(renderer.mlp.b)})
    if getattr(renderer, "vis_sh", None) is not None:
        targets["vis_sh"] = renderer.vis_sh
    missing = sorted(set(targets) - set(sd))
    unexpected = sorted(set(sd) - set(targets))
    if missing or unexpected:
        raise ValueError(f"checkpoint keys differ: missing {missing}, unexpected {unexpected}")
    for k, t in targets.items():
        if tuple(sd[k].shape) != tuple(t.shape):
            raise ValueError(f"checkpoint entry {k}: shape {tuple(sd[k].shape)}, expected {tuple(t.shape)}")
    with torch.no_grad():
        for k, t in targets.items():
            t.copy_(sd[k].to(dtype=t.dtype), non_blocking=False)


def save_checkpoint(path, renderer, step: int = 0, extra: dict | None = None) -> None:
    """Write the renderer's trainable state with the step counter and any
    caller state (optimizer state_dict, RNG state, ...) under `extra`."""
    torch.save({"format": CHECKPOINT_FORMAT, "step": int(step), "state": state_dict(renderer),
                "extra": extra or {}}, path)


def load_checkpoint(path, renderer) -> dict:
    """Restore a checkpoint written by save_checkpoint into `renderer` (in
    place); returns {"step": ..., "extra": ...}. The file is unpickled: load
    only checkpoints you wrote."""
    ck = torch.load(path, map_location="cpu", weights_only=False)
    if not isinstance(ck, dict) or ck.get("format") != CHECKPOINT_FORMAT:
        raise ValueError(f"{path}: not a {CHECKPOINT_FORMAT} file")
    load_state_dict(renderer, ck["state"])
    return {"step": ck["step"], "extra": ck["extra"]}
