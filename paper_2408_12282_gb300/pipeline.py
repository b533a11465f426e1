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


class Renderer:
    """Owns every buffer of a batch and runs the forward/backward call sequence."""

    def __init__(self, scene: dict, mlp: MLPParams, table: PairTable, cfg: B.Cfg, capacity: int | None = None,
                 fused: bool = True, device="cuda", vis_sh=None, shading: str = "deferred"):
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
        self.grads = {k: torch.zeros_like(v) for k, v in scene.items()}
        self.dW = [torch.zeros_like(w) for w in mlp.W]
        self.db = [torch.zeros_like(b) for b in mlp.b]
        self.vis_item = self.dvis_item = self.dvis_sh = None
        self.vis_traced = None
        self.loss_vis = None
        if vis_sh is not None:
            self.vis_item = torch.zeros(n, **f32)
            self.dvis_item = torch.zeros(n, **f32)
            self.dvis_sh = torch.zeros_like(vis_sh)
        self._scene_s = B.scene_struct(scene, self.vis_item)
        self._grad_s = B.scene_grad_struct(self.grads, self.dvis_item)
        self._mlp_s = mlp.struct()
        self._mlp_g = B.mlp_grad_struct(self.dW, self.db)
        mws = B.mlp_workspace_bytes(self._mlp_s, n)
        self.ws_mlp = torch.empty(max(mws, 256), device=device, dtype=torch.uint8)
        self.stats_fwd = None        # optional uint64[2] work counters (see sssgs_render_fwd/bwd)
        self.stats_bwd = None
        self.capacity = 0
        self.set_capacity(capacity if capacity is not None else max(1024, 16 * n))

    # ------------------------------------------------------------------ setup
    def set_capacity(self, cap: int):
        cap = int(cap)
        self.capacity = cap
        self.vals = torch.zeros(max(cap, 1), device=self.device, dtype=torch.int32)
        wsb = B.bin_workspace_bytes(self.table.n_items, cap, self.table.n_tiles)
        self.ws_bin = torch.empty(max(wsb, 256), device=self.device, dtype=torch.uint8)

    def fit_capacity(self, slack: float = 1.15):
        """Run the front end once and size the instance buffers (syncs)."""
        self.forward_front()
        torch.cuda.synchronize()
        need = int(self.count.item())
        if need > self.capacity or self.status.item() != 0:
            self.set_capacity(int(need * slack) + 1024)
            self.status.zero_()
            self.forward_front()
            torch.cuda.synchronize()
        return need

    # ------------------------------------------------------------------ steps
    def forward_front(self, stream=None):
        t = self.table
        if self.vis_sh is not None:
            B.vis_sh_fwd(t.h, t.d, self._scene_s, self.vis_sh, self.vis_item, stream)
        B.mlp_fwd(self._mlp_s, t.h, t.d, self._scene_s, self.mlp_out, self.status, stream)
        B.project_fwd(self.cfg, t.h, t.d, self._scene_s, self.mlp_out, self.rec, self.rect, stream)
        B.bin_sort(self.cfg, t.h, t.d, self.rec, self.rect, self.capacity, self.vals, self.ranges, self.count,
                   self.status, self.ws_bin, stream)

    def forward(self, stream=None):
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
        for g in self.grads.values():
            g.zero_()
        for g in self.dW + self.db:
            g.zero_()
        if self.vis_sh is not None:
            self.dvis_item.zero_()
            self.dvis_sh.zero_()

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
            raise B.SSSGSError(f"instance capacity {self.capacity} exceeded ({int(self.count.item())} needed)")
        if s & B.STATUS_TIMEOUT:
            raise B.SSSGSError("a tensor-core kernel stopped on its wait limit; outputs are incomplete")


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
                          pair_slice=None, vis_sh=None, shading="deferred") -> Renderer:
    """vis_sh: optional N x 16 numpy array of SH visibility coefficients."""
    cfg = default_cfg(tile or wl.tile)
    scene, offs, counts = concat_scenes(wl.scenes, device)
    pairs = wl.pairs if pair_slice is None else wl.pairs[pair_slice]
    table = PairTable(pairs, cfg, offs, counts, device)
    mlp = mlp_to_device(wl.mlp, precision, device)
    sh = None
    if vis_sh is not None:
        sh = torch.from_numpy(np.ascontiguousarray(vis_sh, np.float32)).to(device)
    return Renderer(scene, mlp, table, cfg, capacity=capacity, fused=fused, device=device, vis_sh=sh,
                    shading=shading)


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
        self.grads = {k: torch.zeros_like(v) for k, v in scene.items()}
        self.dW = [torch.zeros_like(w) for w in mlp.W]
        self.db = [torch.zeros_like(b) for b in mlp.b]
        self.vis_sh = vis_sh
        self.vis_item = self.dvis_item = self.dvis_sh = self.vis_traced = self.loss_vis = None
        if vis_sh is not None:
            self.vis_item = torch.zeros(npi, **f32)
            self.dvis_item = torch.zeros(npi, **f32)
            self.dvis_sh = torch.zeros_like(vis_sh)
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
        for g in self.grads.values():
            g.zero_()
        for g in self.dW + self.db:
            g.zero_()
        if self.vis_sh is not None:
            self.dvis_item.zero_()
            self.dvis_sh.zero_()

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


def autotune_tile(wl, candidates=(16, 8), precision=None, steps=2, device="cuda", capacity_slack=1.15):
    """Pick the tile edge for a workload by timing full forward + backward steps
    of each candidate on the device (CUDA events). Returns (best_tile, {tile: ms})."""
    timings = {}
    for tile in candidates:
        r = renderer_for_workload(wl, precision=precision, tile=tile, device=device)
        r.fit_capacity(capacity_slack)
        dimg = torch.full((r.table.n_pixels, 3), 1e-6, device=device)
        r.forward()
        r.backward(dimg=dimg)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            r.forward()
            r.backward(dimg=dimg)
        e1.record()
        torch.cuda.synchronize()
        timings[tile] = e0.elapsed_time(e1) / steps
        del r
        torch.cuda.empty_cache()
    best = min(timings, key=timings.get)
    return best, timings


# ---------------------------------------------------------------------- data parallel

def shard_pairs(n_pairs: int, rank: int, world: int) -> list:
    """Pairs owned by `rank` when a batch of view/light pairs is split over
    `world` processes (round-robin, so uneven batches stay balanced)."""
    return list(range(rank, n_pairs, world))


def allreduce_gradients(tensors, group=None):
    """Sum gradients over the process group: the one exchange of a
    data-parallel step (renders of different pairs are independent; the
    parameters are shared)."""
    import torch.distributed as dist
    for t in tensors:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)


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
