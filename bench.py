#!/usr/bin/env python
"""Throughput of the differentiable OLAT render (forward + backward).

Default workload: the 300K-Gaussian blob scene with 64 view/light pairs at
800x800 (cameras on a radius-3 hemisphere, lights on a radius-4 sphere, both
Fibonacci lattices), 16x16 tiles, PE6 network with four 128-wide layers. One
step = network forward, projection, bin + sort, fused composite + shade, L1
loss gradient against a target image, fused shade + composite backward,
network backward and projection backward, for all 64 pairs.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0). Under torchrun each rank renders its own
64-pair batch (weak scaling) and the parameter gradients are summed with one
NCCL all-reduce per step.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+bwd view-light renders/sec and % HBM roofline vs plain FP32 path at ≤1e-4 err"
UNIT = "renders/s"
L2_BYTES = 129 * 2 ** 20


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), float(d.get("bf16_tflops_sustained", d["bf16_tflops"])), "measured"
    except Exception:
        return 6800.0, 1900.0, 1700.0, "fallback"


# ---------------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.lines = []
        self.proc = None
        self.uuid = uuid

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------- CPU oracle sample

_CPU_SAMPLE = r"""
import json, sys, time
sys.path.insert(0, ROOT)
import numpy as np
import scenegen as sg, oracle as O
wl = sg.make_workload(WORKLOAD, net=NET)
pair = wl.pairs[0]
sc = wl.scenes[pair.scene]
stride = STRIDE
pix = O.all_pixels(pair.W, pair.H)
sel = pix[(pix[:, 1] % stride == 0)]
dimg = sg.random_dimg(7, sel.shape[0])
O.lib()
t0 = time.perf_counter()
X = O.mlp_inputs(wl.mlp.kind, sc.mu, sc.normal, sc.vis, pair.center, pair.light, sc.quat, sc.log_s)
acts, y, Ls, Lin = O.mlp_forward(wl.mlp, X)
dW = O.mlp_backward(wl.mlp, acts, y, Ls, np.ones_like(Ls), np.ones_like(Lin))
t_mlp = time.perf_counter() - t0
t0 = time.perf_counter()
r = O.render_pair(sc, pair, wl.mlp, pixels=sel.astype(np.int32), dimg=dimg)
t_all = time.perf_counter() - t0
t_raster = max(t_all - t_mlp, 1e-9)
full = t_mlp + t_raster * stride
print(json.dumps({"t_mlp": t_mlp, "t_sample": t_all, "t_full_est": full, "pixels": int(sel.shape[0])}))
"""


def cpu_oracle_sample(workload: str, stride: int, threads: int, net=None):
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(threads)
    env["CUDA_VISIBLE_DEVICES"] = ""
    code = (_CPU_SAMPLE.replace("ROOT", repr(ROOT)).replace("WORKLOAD", repr(workload)).replace("STRIDE", str(stride))
            .replace("NET", repr(net)))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


# ---------------------------------------------------------------------------- reference arm

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    threads = os.cpu_count() or 1
    stride = 16
    times = []
    for i in range(args.warmup + args.steps):
        d = cpu_oracle_sample(args.workload, stride, threads, args.net)
        if i >= args.warmup:
            times.append(d["t_full_est"])
    t = sum(times) / len(times)
    value = 1.0 / t
    sample = (f"one view/light pair of workload {args.workload}: full network fwd+bwd over all Gaussians "
              f"(numpy, {threads} BLAS threads), raster fwd+bwd on every {stride}th pixel row (C, one thread), "
              f"raster time scaled by {stride}")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * t, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _config(args),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _config(args):
    desc = {
        "c4": "300K Gaussians on a seeded SH blob, 64 view/light pairs at 800x800 (Fibonacci cameras r=3 "
              "hemisphere, lights r=4 sphere), PE6 MLP 64-128x4-4",
        "c3": "300K Gaussians on a seeded SH blob, 1 view/light pair at 800x800, PE6 MLP 64-128x4-4",
        "c2": "100K Gaussians on a seeded SH blob, 1 pair at 512x512, MLP 9-64x3-4",
        "c1": "1,024 Gaussians in a shell, 1 pair at 128x128, MLP 9-32x2-4",
        "c5": "8 blob scenes of 50K-1M Gaussians x 8 view/light pairs each, resolutions drawn from "
              "{400,800,1200,1600}^2, PE6 MLP 64-128x4-4",
        "c6": "300K Gaussians on the c3 blob, light-stage batch: 8 views (Fibonacci cameras r=3 hemisphere) x "
              "8 lights each of the 112-light stage (7 rings x 16, r=4 upper hemisphere), 800x800, PE6 MLP "
              "64-128x4-4; geometry shared by the lights of a view",
    }
    cfg = {"workload": f"{args.workload}: {desc.get(args.workload, args.workload)}", "tile": args.tile,
           "loss": ("App. E: 0.8 L1 + 0.2 D-SSIM vs target rendered from perturbed parameters "
                    "+ 0.02 incident-light constraint" if args.loss == "paper"
                    else "L1 vs target rendered from perturbed parameters"),
           "l2": "inputs larger than L2 (G-buffer and instance lists >> 129 MB)"}
    if args.pairs is not None:
        cfg["pairs_override"] = args.pairs
    if getattr(args, "shading", "deferred") == "gaussian":
        cfg["shading"] = "per Gaussian (the paper's w/o-Deferred ablation), App. E losses"
    if getattr(args, "vis_sh", False):
        cfg["visibility"] = ("SH term per Gaussian (degree 3, evaluated at each pair's light direction) with the "
                             "ray-traced visibility loss (0.01 L1 to a BVH-traced target)")
    if getattr(args, "views", None) is not None:
        cfg["views_override"] = args.views
    if getattr(args, "lights", None) is not None:
        cfg["lights_override"] = args.lights
    if args.net is not None:
        cfg["network"] = ("the paper's network (App. E): 42 inputs padded to 48, Leaky-ReLU trunk 64-32-32, "
                          "incident head 32-1, SSS head 3, FP32 CUDA cores")
    return cfg


# ---------------------------------------------------------------------------- our arm

STAGES = ("mlp_fwd", "project_fwd", "bin_sort", "render_fwd", "render_bwd", "mlp_bwd", "project_bwd")


def algorithmic_bytes(stage, n_items, n_pixels, n_inst, n_gauss, n_pairs):
    """Compulsory (algorithmic) bytes per launch of each stage."""
    if stage == "render_fwd":          # gbuf 64 + last 4 + img 12 per pixel; id 4 per instance; record 96 per item
        return 80 * n_pixels + 4 * n_inst + 96 * n_items
    if stage == "render_bwd":          # gbuf 64 + last 4 + img 12 + target 12 per pixel; id 4; record 96 + grad 84
        return 92 * n_pixels + 4 * n_inst + 180 * n_items
    if stage == "project_fwd":         # params 84 + net out 16 -> record 96 + rect 16
        return 212 * n_items
    if stage == "project_bwd":         # grad record 96 + net-input grad 28 per item; params 84 + grads 84 rw
        return 124 * n_items + 252 * n_gauss
    if stage == "bin_sort":            # key+id write 12, one read+write pass 24, per instance; depth keys per item
        return 36 * n_inst + 32 * n_items
    if stage == "mlp_fwd":
        return 44 * n_items
    if stage == "mlp_bwd":
        return 72 * n_items
    return 0


# FP32 operations per unit of the fused render kernels (counted from the kernel
# source: an alpha evaluation, a composited contribution, the per-pixel
# shading and its backward; an FMA counts 2)
FLOP_EVAL = 14
FLOP_FWD_CONTRIB = 47
FLOP_BWD_CONTRIB = 105
FLOP_SHADE_FWD = 120
FLOP_SHADE_BWD = 300
ALU_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


# DRAM bytes (read + write) per 300K / 800x800 pair of the fused render kernels,
# from one ncu capture of an 8-pair launch of the same scene
# (profiles/k_composite_*_warp_300k_800_8pairs.md), divided by 8. Valid only
# for the kernel sources they were taken on (sha256 of raster.cu followed by
# raster_common.cuh) and for workloads made of such pairs; otherwise null.
TRAFFIC_SOURCES = ("raster.cu", "raster_common.cuh")
KERNEL_TRAFFIC = {
    "render_bwd": ("5d56c5a2c34af8132c2dbc4eff46949b4f7e384f5a34f41e2b28c9948bb5a861", 108.68e6),
    "render_fwd": ("5d56c5a2c34af8132c2dbc4eff46949b4f7e384f5a34f41e2b28c9948bb5a861", 70.47e6),
}


def render_source_sha():
    import hashlib
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2408_12282_gb300", "csrc", f),
                  "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def kernel_traffic(stage, workload, n_pairs):
    if stage not in KERNEL_TRAFFIC or workload not in ("c3", "c4"):
        return None
    sha, per_pair = KERNEL_TRAFFIC[stage]
    if render_source_sha() != sha:
        return None
    return per_pair * n_pairs


def mlp_flops(widths, rows):
    f = 0
    for a, b in zip(widths[:-1], widths[1:]):
        f += 2 * a * b
    return f * rows


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import scenegen as sg
    from paper_2408_12282_gb300 import binding as B
    from paper_2408_12282_gb300 import pipeline as PL

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    B.load_library()
    hbm, bf16_burst, bf16_sus, peak_src = _peaks()

    wl = sg.make_workload(args.workload, seed_offset=rank, n_pairs=args.pairs, net=args.net)
    precision = B.BF16 if (wl.mlp.precision == "bf16" and not args.fp32_mlp) else B.FP32
    vis_sh = sg.vis_sh_coeffs(77 + rank, sum(sc.N for sc in wl.scenes)) if args.vis_sh else None
    r = PL.renderer_for_workload(wl, precision=precision, tile=args.tile, vis_sh=vis_sh, shading=args.shading)
    n_inst = r.fit_capacity()
    trace = None
    if args.vis_sh:
        # ray-traced visibility target (BVH build + one ray per item), timed once
        r.trace_visibility()
        torch.cuda.synchronize()
        tb0, tb1, tt1 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        tb0.record()
        B.bvh_build(r.cfg, r._scene_s, r.bvh, r.ws_bvh)
        tb1.record()
        B.trace_visibility(r.cfg, r.table.h, r.table.d, r._scene_s, r.bvh, r.vis_traced)
        tt1.record()
        torch.cuda.synchronize()
        tms = tb1.elapsed_time(tt1)
        trace = {"rays": r.table.n_items, "bvh_build_ms": tb0.elapsed_time(tb1), "trace_ms": tms,
                 "rays_per_s": r.table.n_items * 1000.0 / tms,
                 "mean_visibility": float(r.vis_traced.mean().item())}
    table = r.table
    n_pairs = table.n
    # target images from the perturbed scene (untimed set-up)
    tgt_scenes = ([wl.target_scene] if wl.target_scene is not None and len(wl.scenes) == 1 else
                  [sg.perturbed(s, 4242 + 97 * rank + i) for i, s in enumerate(wl.scenes)])
    wl_t = sg.Workload(wl.name, tgt_scenes, wl.pairs, wl.mlp, wl.tile)
    rt = PL.renderer_for_workload(wl_t, precision=precision, tile=args.tile)
    rt.fit_capacity()
    rt.forward()
    target = rt.img.clone()
    del rt
    torch.cuda.empty_cache()
    l1_scale = 1.0 / (3.0 * table.n_pixels)
    grads_flat = [g for g in r.grads.values()] + r.dW + r.db

    graph = None
    graph_launches = 0
    if not args.no_graph:
        c0 = B.launch_count()
        graph = r.capture(target=target, l1_scale=l1_scale, loss=args.loss)
        graph_launches = (B.launch_count() - c0) // 2      # capture() runs the step once eagerly, once captured

    def step():
        if graph is not None:
            graph.replay()
        else:
            r.forward()
            r.backward(target=target, l1_scale=l1_scale, loss=args.loss)
        if world > 1:
            PL.allreduce_gradients(grads_flat)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    r.check_status()

    # ---------------- timed region (device events on the launching stream)
    st = torch.cuda.current_stream()
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        uuid = None
    sampler = ClockSampler(uuid)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    l0 = B.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        step()
    e1.record(st)
    torch.cuda.synchronize()
    launches = graph_launches if graph is not None else (B.launch_count() - l0) // args.steps
    clocks = sampler.stop()
    if world > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1) / args.steps
    ms_t = torch.tensor([ms], device="cuda")
    if world > 1:
        dist.all_reduce(ms_t, op=dist.ReduceOp.MAX)
    ms_max = float(ms_t.item())
    value = world * n_pairs * 1000.0 / ms_max

    # ---------------- per-stage timing (separate pass, events between calls)
    stages = STAGES + (("loss",) if args.loss == "paper" else ())
    stage_ms = {s: 0.0 for s in stages}
    reps = max(2, min(args.steps, 5))
    stats_f = torch.zeros(2, dtype=torch.int64, device="cuda")
    stats_b = torch.zeros(2, dtype=torch.int64, device="cuda")
    if args.vis_sh:
        stage_ms["vis_sh"] = 0.0
    for _ in range(reps if args.shading == "deferred" else 0):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(STAGES) + 1)]
        ev_v = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        if args.vis_sh:
            ev_v[0].record(st)
            B.vis_sh_fwd(table.h, table.d, r._scene_s, r.vis_sh, r.vis_item)
            ev_v[1].record(st)
        ev[0].record(st)
        B.mlp_fwd(r._mlp_s, table.h, table.d, r._scene_s, r.mlp_out, r.status)
        ev[1].record(st)
        B.project_fwd(r.cfg, table.h, table.d, r._scene_s, r.mlp_out, r.rec, r.rect)
        ev[2].record(st)
        B.bin_sort(r.cfg, table.h, table.d, r.rec, r.rect, r.capacity, r.vals, r.ranges, r.count, r.status, r.ws_bin)
        ev[3].record(st)
        B.render_fwd(r.cfg, table.h, table.d, r.rec, r.vals, r.ranges, r.gbuf, r.last, r.img, stats_f)
        ev[4].record(st)
        r.zero_grads()
        e_z = torch.cuda.Event(enable_timing=True)
        e_l = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        if args.loss == "paper":
            e_l[0].record(st)
            r.loss.zero_()
            B.image_loss(r.cfg, table.h, table.d, r.img, target, 0.2, r.dimg_loss, r.loss, r.ws_loss)
            e_l[1].record(st)
        e_z.record(st)
        if args.loss == "paper":
            B.render_bwd(r.cfg, table.h, table.d, r.rec, r.vals, r.ranges, r.gbuf, r.last, r.img, r.dimg_loss,
                         None, None, 1.0, r.drec, stats_b)
            e_l[2].record(st)
            B.incident_loss(table.h, table.d, r.rec, 0.02, r.drec, r.loss)
            e_l[3].record(st)
        else:
            B.render_bwd(r.cfg, table.h, table.d, r.rec, r.vals, r.ranges, r.gbuf, r.last, r.img, None, target,
                         None, l1_scale, r.drec, stats_b)
        ev[5].record(st)
        B.mlp_bwd(r._mlp_s, table.h, table.d, r._scene_s, r.drec, r._mlp_g, r.dx_items, r.ws_mlp, r.status)
        ev[6].record(st)
        B.project_bwd(r.cfg, table.h, table.d, r._scene_s, r.drec, r.dx_items, r._grad_s)
        ev[7].record(st)
        if args.vis_sh:
            ev_v[2].record(st)
            r.loss_vis = r.loss_vis if r.loss_vis is not None else torch.zeros(table.n, device="cuda")
            B.vis_loss(table.h, table.d, r.vis_item, r.vis_traced, 0.01, r.dvis_item, r.loss_vis)
            B.vis_sh_bwd(table.h, table.d, r._scene_s, r.vis_sh, r.dvis_item, r.dvis_sh, r.grads["mu"])
            ev_v[3].record(st)
        torch.cuda.synchronize()
        if args.vis_sh:
            stage_ms["vis_sh"] += (ev_v[0].elapsed_time(ev_v[1]) + ev_v[2].elapsed_time(ev_v[3])) / reps
        for i, s in enumerate(STAGES):
            a = e_z if s == "render_bwd" else ev[i]
            b = e_l[2] if (s == "render_bwd" and args.loss == "paper") else ev[i + 1]
            stage_ms[s] += a.elapsed_time(b) / reps
        if args.loss == "paper":
            stage_ms["loss"] += (e_l[0].elapsed_time(e_l[1]) + e_l[2].elapsed_time(e_l[3])) / reps
    if args.shading == "gaussian":      # the ablation path: forward and backward timed as wholes
        stage_ms = {"forward": 0.0, "backward": 0.0}
        for _ in range(reps):
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record(st)
            r.forward()
            e[1].record(st)
            r.backward(target=target, loss="paper")
            e[2].record(st)
            torch.cuda.synchronize()
            stage_ms["forward"] += e[0].elapsed_time(e[1]) / reps
            stage_ms["backward"] += e[1].elapsed_time(e[2]) / reps
        for k in STAGES:
            stage_ms.setdefault(k, 0.0)
    n_items, n_pixels = table.n_items, table.n_pixels
    # rows the network backward runs on: items with a nonzero upstream gradient
    # (the others add exactly zero and are compacted out)
    n_active = int((r.drec[:, 16:20] != 0).any(dim=1).sum().item())
    n_gauss = sum(sc.N for sc in wl.scenes)
    contrib_f, evals_f = (int(x) // reps for x in stats_f.tolist())
    contrib_b, evals_b = (int(x) // reps for x in stats_b.tolist())
    alu_flops = {
        "render_fwd": FLOP_FWD_CONTRIB * contrib_f + FLOP_EVAL * (evals_f - contrib_f) + FLOP_SHADE_FWD * n_pixels,
        "render_bwd": FLOP_BWD_CONTRIB * contrib_b + FLOP_EVAL * (evals_b - contrib_b) + FLOP_SHADE_BWD * n_pixels,
    }
    dom = max(STAGES, key=lambda s: stage_ms[s])
    widths = [int(r._mlp_s.width[i]) for i in range(r._mlp_s.n_layers + 1)]
    if args.shading == "gaussian":      # an ablation configuration: stages are not split
        roof = None
    elif dom in ("mlp_fwd", "mlp_bwd") and precision == B.BF16:
        fl = mlp_flops(widths, n_items) if dom == "mlp_fwd" else 2 * mlp_flops(widths, n_active)
        ach = fl / (stage_ms[dom] * 1e-3) / 1e12
        roof = {"bound": "tensor", "kernel": dom, "achieved": ach, "peak": bf16_sus, "unit": "TFLOP/s",
                "frac": ach / bf16_sus, "traffic": None, "peak_source": peak_src + " (bf16 sustained)"}
    elif dom in alu_flops:
        ach = alu_flops[dom] / (stage_ms[dom] * 1e-3) / 1e12
        roof = {"bound": "alu", "kernel": dom, "achieved": ach, "peak": ALU_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / ALU_PEAK_TFLOPS, "traffic": kernel_traffic(dom, args.workload, n_pairs),
                "traffic_unit": "DRAM bytes per launch (ncu on an 8-pair launch, scaled per pair)",
                "peak_source": "152 SMs x 128 FP32 lanes x 2 FLOP x 2.07 GHz",
                "work": {"contributions": contrib_b if dom == "render_bwd" else contrib_f,
                         "alpha_evaluations": evals_b if dom == "render_bwd" else evals_f},
                "hbm_frac_of_algorithmic_bytes": algorithmic_bytes(dom, n_items, n_pixels, n_inst, n_gauss, n_pairs)
                / (stage_ms[dom] * 1e-3) / 1e9 / hbm}
    else:
        by = algorithmic_bytes(dom, n_items, n_pixels, n_inst, n_gauss, n_pairs)
        ach = by / (stage_ms[dom] * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "traffic": None, "peak_source": peak_src + " (hbm copy)"}
    total_bytes = sum(algorithmic_bytes(s, n_items, n_pixels, n_inst, n_gauss, n_pairs) for s in STAGES)
    loss_roof = None
    if args.loss == "paper" and "loss" in stage_ms:
        # SSIM pass A: img + target in, 9 coefficient floats out; pass B: the
        # coefficients + img + target in, dimg out; incident: L_in, v in and
        # their two gradient slots read-modify-written
        by = 132 * n_pixels + 24 * n_items
        ach = by / (stage_ms["loss"] * 1e-3) / 1e9
        loss_roof = {"bound": "hbm", "kernels": "k_ssim_moments + k_ssim_grad + k_incident", "achieved": ach,
                     "peak": hbm, "unit": "GB/s", "frac": ach / hbm, "algorithmic_bytes": by}
    step_hbm_frac = total_bytes / (ms_max * 1e-3) / 1e9 / hbm

    # ---------------- plain unbatched FP32 path (per-pair launches, unfused, CUDA-core network)
    plain = None
    if not args.skip_plain:
        k = min(args.plain_pairs, n_pairs)
        rp = PL.renderer_for_workload(wl, precision=B.FP32, fused=False, tile=args.tile, pair_slice=slice(0, 1))
        rp.fit_capacity()
        rp.set_capacity(int(1.5 * n_inst / n_pairs) + 4096)
        tables = [PL.PairTable([wl.pairs[i]], rp.cfg, [0], [n_gauss]) for i in range(k)]
        dimg_p = torch.full((rp.table.n_pixels, 3), l1_scale, device="cuda")

        def plain_step():
            for tb in tables:
                rp.table = tb
                rp.forward()
                rp.backward(dimg=dimg_p)
        plain_step()
        torch.cuda.synchronize()
        p0 = torch.cuda.Event(enable_timing=True)
        p1 = torch.cuda.Event(enable_timing=True)
        p0.record(st)
        plain_step()
        p1.record(st)
        torch.cuda.synchronize()
        pms = p0.elapsed_time(p1)
        plain = {"renders_per_s": k * 1000.0 / pms, "pairs_timed": k,
                 "what": "per-pair launches, unfused composite and shade, FP32 CUDA-core network",
                 "speedup_of_batched": value / world / (k * 1000.0 / pms)}
        del rp
        torch.cuda.empty_cache()

    # ---------------- end to end through the public API with host buffers
    e2e = None
    if not args.skip_e2e:
        host_in = {k: v.detach().cpu().pin_memory() for k, v in r.scene.items()}
        host_tgt = target.cpu().pin_memory()
        host_out = {k: torch.empty_like(v, device="cpu").pin_memory() for k, v in r.grads.items()}
        h2d = sum(v.numel() * 4 for v in host_in.values()) + host_tgt.numel() * 4
        d2h = sum(v.numel() * 4 for v in host_out.values())
        loss_host = None
        if args.loss == "paper":
            loss_host = torch.empty(n_pairs, dtype=torch.float32).pin_memory()
            d2h += n_pairs * 4

        def e2e_step():
            for k2, v in host_in.items():
                r.scene[k2].copy_(v, non_blocking=True)
            target.copy_(host_tgt, non_blocking=True)
            if graph is not None:
                graph.replay()
            else:
                r.forward()
                r.backward(target=target, l1_scale=l1_scale, loss=args.loss)
            if world > 1:
                PL.allreduce_gradients(grads_flat)
            if loss_host is not None:
                loss_host.copy_(r.loss, non_blocking=True)
            for k2, v in host_out.items():
                v.copy_(r.grads[k2], non_blocking=True)
        for _ in range(args.warmup):       # same warm-up as the device-timed loop
            e2e_step()
        torch.cuda.synchronize()
        q0 = torch.cuda.Event(enable_timing=True)
        q1 = torch.cuda.Event(enable_timing=True)
        q0.record(st)
        for _ in range(args.steps):
            e2e_step()
        q1.record(st)
        torch.cuda.synchronize()
        ems = q0.elapsed_time(q1) / args.steps
        e2e = {"value": world * n_pairs * 1000.0 / ems, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}

    # ---------------- CPU oracle baseline (rank 0, one GPU only)
    cpu = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        try:
            d = cpu_oracle_sample(args.workload, 16, 1, args.net)
            cpu = {"value": 1.0 / d["t_full_est"], "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": (f"one pair of {args.workload}: network fwd+bwd over all {n_gauss} Gaussians "
                              f"({d['t_mlp']:.1f} s) + raster fwd+bwd on every 16th pixel row "
                              f"({d['t_sample'] - d['t_mlp']:.1f} s) scaled by 16; single thread")}
        except Exception as ex:  # report, do not hide
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": f"failed: {ex}"[:300]}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "bf16+f32" if precision == B.BF16 else "f32",
                "data": "synthetic", "config": _config(args),
                "roofline": roof, "step_hbm_frac_of_algorithmic": step_hbm_frac,
                "stage_ms": stage_ms, "loss_roofline": loss_roof, "visibility_trace": trace, "instances": n_inst, "items": n_items, "mlp_bwd_rows": n_active, "pixels": n_pixels,
                "contributions_per_step": {"forward": contrib_f, "backward": contrib_b},
                "cuda_graph": graph is not None,
                "plain_fp32": plain, "e2e": e2e, "gpu_launches": int(launches), "clocks": clocks,
                "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------- many lights per view

def ml_alu_flops(L, contrib_f, evals_f, contrib_b, evals_b, view_pixels):
    """FP32 operations of the many-light render kernels: per contribution the
    single-light count plus, per further light, 4 composited channels (fwd: 4
    FMA; bwd: 4 FMA in the dot product, 4 products and 4 reduction adds), and
    the shading (and its backward) once per light and view pixel."""
    fwd = ((FLOP_FWD_CONTRIB + 8 * (L - 1)) * contrib_f + FLOP_EVAL * (evals_f - contrib_f)
           + FLOP_SHADE_FWD * L * view_pixels)
    bwd = ((FLOP_BWD_CONTRIB + 16 * (L - 1)) * contrib_b + FLOP_EVAL * (evals_b - contrib_b)
           + FLOP_SHADE_BWD * L * view_pixels)
    return {"render_fwd": fwd, "render_bwd": bwd}


def run_ours_ml(args):
    """Light-stage batches (workload c6): n_views views x n_lights lights, one
    step = forward + backward of every (view, light) pair, the geometry shared
    by the lights of a view (MultiLightRenderer). Also times the single-light
    batched path on the same pairs for comparison."""
    import torch
    import torch.distributed as dist

    import scenegen as sg
    from paper_2408_12282_gb300 import binding as B
    from paper_2408_12282_gb300 import pipeline as PL

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    B.load_library()
    hbm, bf16_burst, bf16_sus, peak_src = _peaks()
    wl = sg.make_workload(args.workload, seed_offset=rank, net=args.net, n_views=args.views, n_lights=args.lights)
    precision = B.BF16 if (wl.mlp.precision == "bf16" and not args.fp32_mlp) else B.FP32
    L = wl.n_lights
    r = PL.multilight_renderer_for_workload(wl, precision=precision)
    n_inst = r.fit_capacity()
    n_pairs = len(wl.pairs)
    wl_t = sg.Workload(wl.name, [sg.perturbed(s, 4242 + 97 * rank) for s in wl.scenes], wl.pairs, wl.mlp, wl.tile,
                       None, n_lights=L)
    rt = PL.multilight_renderer_for_workload(wl_t, precision=precision)
    rt.fit_capacity()
    rt.forward()
    target = rt.img.clone()
    del rt
    torch.cuda.empty_cache()
    l1_scale = 1.0 / (3.0 * r.pairs.n_pixels)
    grads_flat = [g for g in r.grads.values()] + r.dW + r.db
    c0 = B.launch_count()
    graph = r.capture(target=target, l1_scale=l1_scale)
    graph_launches = (B.launch_count() - c0) // 2

    def step():
        graph.replay()
        if world > 1:
            PL.allreduce_gradients(grads_flat)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    r.check_status()
    st = torch.cuda.current_stream()
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        uuid = None
    sampler = ClockSampler(uuid)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        step()
    e1.record(st)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    if world > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1) / args.steps
    ms_t = torch.tensor([ms], device="cuda")
    if world > 1:
        dist.all_reduce(ms_t, op=dist.ReduceOp.MAX)
    ms_max = float(ms_t.item())
    value = world * n_pairs * 1000.0 / ms_max

    # per-stage timing (separate pass)
    stages = ("mlp_fwd", "project_fwd", "bin_sort", "render_fwd", "render_bwd", "mlp_bwd", "project_bwd")
    stage_ms = {k: 0.0 for k in stages}
    reps = max(2, min(args.steps, 5))
    r.stats_fwd = torch.zeros(2, dtype=torch.int64, device="cuda")
    r.stats_bwd = torch.zeros(2, dtype=torch.int64, device="cuda")
    v, pt = r.views, r.pairs
    for _ in range(reps):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(9)]
        ev[0].record(st)
        B.mlp_fwd(r._mlp_s, pt.h, pt.d, r._scene_s, r.mlp_out, r.status)
        ev[1].record(st)
        B.project_fwd(r.cfg, v.h, v.d, r._scene_s, None, r.rec, r.rect)
        ev[2].record(st)
        B.bin_sort(r.cfg, v.h, v.d, r.rec, r.rect, r.capacity, r.vals, r.ranges, r.count, r.status, r.ws_bin)
        ev[3].record(st)
        B.render_ml_fwd(r.cfg, v.h, v.d, L, r.lights, r.rec, r.mlp_out, r.vals, r.ranges, r.gbuf, r.last, r.img,
                        None, r.stats_fwd)
        ev[4].record(st)
        r.zero_grads()
        ev[5].record(st)
        B.render_ml_bwd(r.cfg, v.h, v.d, L, r.lights, r.rec, r.mlp_out, r.vals, r.ranges, r.gbuf, r.last, r.img,
                        None, target, l1_scale, r.drec, r.dmlp, r.stats_bwd)
        ev[6].record(st)
        B.mlp_bwd_strided(r._mlp_s, pt.h, pt.d, r._scene_s, r.dmlp, 4, r._mlp_g, r.dx_items, r.ws_mlp, r.status)
        ev[7].record(st)
        B.project_bwd(r.cfg, v.h, v.d, r._scene_s, r.drec, None, r._grad_s)
        B.project_bwd(r.cfg, pt.h, pt.d, r._scene_s, None, r.dx_items, r._grad_s)
        ev[8].record(st)
        torch.cuda.synchronize()
        pairs_ev = [(0, 1), (1, 2), (2, 3), (3, 4), (5, 6), (6, 7), (7, 8)]
        for k, (a, b) in zip(stages, pairs_ev):
            stage_ms[k] += ev[a].elapsed_time(ev[b]) / reps
    contrib_f, evals_f = (int(x) // reps for x in r.stats_fwd.tolist())
    contrib_b, evals_b = (int(x) // reps for x in r.stats_bwd.tolist())
    n_active = int((r.dmlp != 0).any(dim=1).sum().item())
    alu = ml_alu_flops(L, contrib_f, evals_f, contrib_b, evals_b, v.n_pixels)
    dom = max(stages, key=lambda k: stage_ms[k])
    widths = [int(r._mlp_s.width[i]) for i in range(r._mlp_s.n_layers + 1)]
    if dom in ("mlp_fwd", "mlp_bwd") and precision == B.BF16:
        fl = mlp_flops(widths, pt.n_items) if dom == "mlp_fwd" else 2 * mlp_flops(widths, n_active)
        ach = fl / (stage_ms[dom] * 1e-3) / 1e12
        roof = {"bound": "tensor", "kernel": dom, "achieved": ach, "peak": bf16_sus, "unit": "TFLOP/s",
                "frac": ach / bf16_sus, "traffic": None, "peak_source": peak_src + " (bf16 sustained)"}
    elif dom in alu:
        ach = alu[dom] / (stage_ms[dom] * 1e-3) / 1e12
        roof = {"bound": "alu", "kernel": dom + " (many lights)", "achieved": ach, "peak": ALU_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": ach / ALU_PEAK_TFLOPS, "traffic": None,
                "peak_source": "152 SMs x 128 FP32 lanes x 2 FLOP x 2.07 GHz",
                "work": {"contributions": contrib_b if dom == "render_bwd" else contrib_f,
                         "alpha_evaluations": evals_b if dom == "render_bwd" else evals_f, "lights_per_view": L}}
    else:
        roof = {"bound": "hbm", "kernel": dom, "achieved": None, "peak": hbm, "unit": "GB/s", "frac": None,
                "traffic": None, "peak_source": peak_src + " (hbm copy)"}

    # the single-light batched path on the same pairs (each pair on its own)
    single = None
    if not args.skip_plain:
        rs = PL.renderer_for_workload(wl, precision=precision)
        rs.fit_capacity()
        gs = rs.capture(target=target, l1_scale=l1_scale)
        for _ in range(2):
            gs.replay()
        torch.cuda.synchronize()
        p0 = torch.cuda.Event(enable_timing=True)
        p1 = torch.cuda.Event(enable_timing=True)
        p0.record(st)
        for _ in range(args.steps):
            gs.replay()
        p1.record(st)
        torch.cuda.synchronize()
        sms = p0.elapsed_time(p1) / args.steps
        single = {"renders_per_s": n_pairs * 1000.0 / sms, "ms_per_step": sms,
                  "what": "the same pairs through the single-light batched path (geometry per pair)",
                  "speedup_of_many_light": (value / world) / (n_pairs * 1000.0 / sms)}
        del rs, gs
        torch.cuda.empty_cache()

    e2e = None
    if not args.skip_e2e:
        host_in = {k: t.detach().cpu().pin_memory() for k, t in r.scene.items()}
        host_tgt = target.cpu().pin_memory()
        host_out = {k: torch.empty_like(t, device="cpu").pin_memory() for k, t in r.grads.items()}
        h2d = sum(t.numel() * 4 for t in host_in.values()) + host_tgt.numel() * 4
        d2h = sum(t.numel() * 4 for t in host_out.values())

        def e2e_step():
            for k2, t in host_in.items():
                r.scene[k2].copy_(t, non_blocking=True)
            target.copy_(host_tgt, non_blocking=True)
            graph.replay()
            if world > 1:
                PL.allreduce_gradients(grads_flat)
            for k2, t in host_out.items():
                t.copy_(r.grads[k2], non_blocking=True)
        for _ in range(args.warmup):       # same warm-up as the device-timed loop
            e2e_step()
        torch.cuda.synchronize()
        q0 = torch.cuda.Event(enable_timing=True)
        q1 = torch.cuda.Event(enable_timing=True)
        q0.record(st)
        for _ in range(args.steps):
            e2e_step()
        q1.record(st)
        torch.cuda.synchronize()
        ems = q0.elapsed_time(q1) / args.steps
        e2e = {"value": world * n_pairs * 1000.0 / ems, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}

    cpu = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        try:
            d = cpu_oracle_sample(args.workload, 16, 1, args.net)
            cpu = {"value": 1.0 / d["t_full_est"], "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": (f"one view/light pair of {args.workload}: network fwd+bwd over all Gaussians "
                              f"({d['t_mlp']:.1f} s) + raster fwd+bwd on every 16th pixel row "
                              f"({d['t_sample'] - d['t_mlp']:.1f} s) scaled by 16; single thread")}
        except Exception as ex:
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": f"failed: {ex}"[:300]}
    if rank == 0:
        cfg = _config(args)
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "bf16+f32" if precision == B.BF16 else "f32", "data": "synthetic",
                "config": cfg, "roofline": roof, "stage_ms": stage_ms, "instances": n_inst,
                "views": v.n, "lights_per_view": L, "pairs": n_pairs, "mlp_bwd_rows": n_active,
                "contributions_per_step": {"forward": contrib_f, "backward": contrib_b},
                "cuda_graph": True, "single_light_path": single, "e2e": e2e, "gpu_launches": int(graph_launches),
                "clocks": clocks, "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c4")
    ap.add_argument("--net", default=None, choices=[None, "paper"],
                    help="replace the workload's network by the paper's (App. E)")
    ap.add_argument("--pairs", type=int, default=None,
                    help="override the number of view/light pairs (smaller cases for profiling)")
    ap.add_argument("--tile", type=int, default=16)
    ap.add_argument("--views", type=int, default=None, help="c6: views per batch (default 8)")
    ap.add_argument("--lights", type=int, default=None, help="c6: lights per view, 1/2/4/8 (default 8)")
    ap.add_argument("--loss", default="l1", choices=["l1", "paper"],
                    help="paper: the training losses of App. E (L1 + D-SSIM image loss, incident constraint)")
    ap.add_argument("--fp32-mlp", action="store_true")
    ap.add_argument("--shading", default="deferred", choices=["deferred", "gaussian"],
                    help="gaussian: the paper's w/o-Deferred ablation (each Gaussian shaded, colours composited); "
                         "runs with the App. E losses")
    ap.add_argument("--vis-sh", action="store_true",
                    help="SH visibility term per Gaussian (v evaluated at each pair's light) with the ray-traced "
                         "visibility loss; also times the BVH build and the tracing")
    ap.add_argument("--plain-pairs", type=int, default=4)
    ap.add_argument("--skip-plain", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--no-graph", action="store_true")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.shading == "gaussian":
        args.loss = "paper"
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "c6":
        if args.loss != "l1":
            raise SystemExit("c6 (many lights per view) runs the L1 loss")
        run_ours_ml(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
