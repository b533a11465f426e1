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


# ---------------------------------------------------------------------------- CPU leg (the oracle)
#
# The oracle runs only here, in subprocesses on the host cores: (1) the timed
# CPU baseline, (2) the reference arm, (3) the oracle's values at pixels
# sampled from the timed GPU batch, which the bench compares with the batch's
# images (the `parity` object of the JSON line).

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

_CPU_PARITY = r"""
import json, sys, time
sys.path.insert(0, ROOT)
import numpy as np
import scenegen as sg, oracle as O
wl = sg.make_workload(WORKLOAD, net=NET, n_pairs=N_PAIRS)
spec = np.load(SPEC)
out = {}
t0 = time.perf_counter()
for p in spec["pairs"].tolist():
    pr = wl.pairs[p]
    px = np.ascontiguousarray(spec[f"pix_{p}"], np.int32)
    r = O.render_pair(wl.scenes[pr.scene], pr, wl.mlp, pixels=px, bf16=BF16)
    out[f"img_{p}"] = r["img"]
    out[f"margin_{p}"] = r["margin"]
    if BF16:
        out[f"img64_{p}"] = O.render_pair(wl.scenes[pr.scene], pr, wl.mlp, pixels=px)["img"]
np.savez(OUT, **out)
print(json.dumps({"t": time.perf_counter() - t0}))
"""


def _run_cpu(code, threads):
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(threads)
    env["CUDA_VISIBLE_DEVICES"] = ""
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def cpu_oracle_sample(workload: str, stride: int, threads: int, net=None):
    code = (_CPU_SAMPLE.replace("ROOT", repr(ROOT)).replace("WORKLOAD", repr(workload)).replace("STRIDE", str(stride))
            .replace("NET", repr(net)))
    return _run_cpu(code, threads)


def cpu_oracle_pixels(workload: str, net, n_pairs, pixels: dict, bf16: bool):
    """The oracle's image values at the given pixels {pair: (n x 2) int array}
    of the workload (with the BF16-emulating network if bf16, plus the pure
    FP64 network's values), and the decision margins; all host cores."""
    import tempfile
    import numpy as np
    with tempfile.TemporaryDirectory() as td:
        spec = os.path.join(td, "spec.npz")
        res = os.path.join(td, "out.npz")
        np.savez(spec, pairs=np.array(sorted(pixels)), **{f"pix_{p}": v for p, v in pixels.items()})
        code = (_CPU_PARITY.replace("ROOT", repr(ROOT)).replace("WORKLOAD", repr(workload))
                .replace("NET", repr(net)).replace("N_PAIRS", repr(n_pairs)).replace("SPEC", repr(spec))
                .replace("OUT", repr(res))
                .replace("BF16", repr(bool(bf16))))
        t = _run_cpu(code, os.cpu_count() or 1)
        with np.load(res) as z:
            got = {k: z[k] for k in z.files}
    return got, t["t"]


# ---------------------------------------------------------------------------- reference arm

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    threads = os.cpu_count() or 1
    stride = 16
    times, walls = [], []
    for i in range(args.warmup + args.steps):
        w0 = time.perf_counter()
        d = cpu_oracle_sample(args.workload, stride, threads, args.net)
        w1 = time.perf_counter()
        if i >= args.warmup:
            times.append(d["t_full_est"])
            walls.append(w1 - w0)
    t = sum(times) / len(times)
    value = 1.0 / t
    wall = sum(walls) / len(walls)
    sample = (f"one view/light pair of workload {args.workload} per step: full network fwd+bwd over all Gaussians "
              f"(numpy, {threads} BLAS threads) and raster fwd+bwd on every {stride}th pixel row (C, one thread); "
              f"value = 1 / (network time + {stride} x raster-sample time), an extrapolation to a whole render "
              f"({t:.1f} s); ms_per_step is the measured wall time of one sample step (process start and scene "
              f"generation included)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * wall,
            "extrapolated_s_per_render": t, "higher_is_better": True,
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
    tile = ("per scene, autotuned (see schedule)" if args.tile == "auto" and args.shading == "deferred"
            and not getattr(args, "vis_sh", False) else (16 if args.tile == "auto" else int(args.tile)))
    cfg = {"workload": f"{args.workload}: {desc.get(args.workload, args.workload)}", "tile": tile,
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
FLOP_BWD_CONTRIB = 102
FLOP_SHADE_FWD = 120
FLOP_SHADE_BWD = 300
ALU_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


# DRAM bytes (read + write) per 300K / 800x800 pair of the fused render kernels,
# from one ncu capture of an 8-pair launch of the same scene
# (profiles/k_composite_*_warp_300k_800_8pairs.md), divided by 8. Valid only
# for the kernel sources they were taken on (sha256 of raster.cu, then
# raster_common.cuh, then common.cuh) and for workloads made of such pairs;
# otherwise null.
TRAFFIC_SOURCES = ("raster.cu", "raster_common.cuh", "common.cuh")
KERNEL_TRAFFIC = {
    "render_bwd": ("44bf3ed7952819584a2266ec8b961f8bbf2ed8ac7e39a6d083084784cac7165a", 108.33e6),
    "render_fwd": ("44bf3ed7952819584a2266ec8b961f8bbf2ed8ac7e39a6d083084784cac7165a", 81.70e6),
}


def render_source_sha():
    import hashlib
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2408_12282_gb300", "csrc", f),
                  "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def kernel_traffic(stage, workload, n_pairs, tile_batch=(16, 32)):
    """DRAM bytes of one launch of a fused render kernel on this workload:
    only for the kernel source and the schedule (16 x 16 tiles, batches of 32
    splats) the capture was taken on; None otherwise."""
    if stage not in KERNEL_TRAFFIC or workload not in ("c3", "c4") or tuple(tile_batch) != (16, 32):
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


# Parity of the timed batch: pixels whose oracle alpha or stop decision lies
# within this relative distance of its threshold can flip between float32
# and FP64 (a finite jump) and are counted but left out of the gate (the
# margin of the parity tests). Gate: every sampled pixel within 1e-4 of the
# oracle; with the BF16 network against the BF16-emulating oracle, 99.9%
# within 1e-4 and all within 2e-4 (the tests' gate for the batches).
PARITY_FLAG_MARGIN = 1e-4
PARITY_GATE = 1e-4
PARITY_GATE_BF16_MAX = 2e-4


def parity_report(args, n_pairs, par_pix, par_got, bf16):
    import numpy as np
    try:
        ref, t_par = cpu_oracle_pixels(args.workload, args.net, args.pairs, par_pix, bf16)
    except Exception as ex:  # report, do not hide
        return {"error": f"{ex}"[:300]}
    e_all, e64_all, n_flag = [], [], 0
    for p in par_pix:
        rimg = ref[f"img_{p}"]
        m = ref[f"margin_{p}"]
        fl = (m[:, 0] < PARITY_FLAG_MARGIN) | (m[:, 1] < PARITY_FLAG_MARGIN)
        n_flag += int(fl.sum())
        e = (np.abs(par_got[p] - rimg) / np.maximum(1.0, np.abs(rimg))).max(axis=1)
        e_all.append(e[~fl])
        if bf16:
            r64 = ref[f"img64_{p}"]
            e64_all.append((np.abs(par_got[p] - r64) / np.maximum(1.0, np.abs(r64))).max(axis=1)[~fl])
    e = np.concatenate(e_all)
    p999 = float(np.quantile(e, 0.999))
    ok = (p999 <= PARITY_GATE and e.max() <= PARITY_GATE_BF16_MAX) if bf16 else e.max() <= PARITY_GATE
    out = {"pairs": sorted(par_pix), "pixels": int(sum(len(v) for v in par_pix.values())),
           "flag_margin": PARITY_FLAG_MARGIN, "flagged": n_flag,
           "gate": (f"p99.9 <= {PARITY_GATE}, max <= {PARITY_GATE_BF16_MAX}" if bf16 else f"max <= {PARITY_GATE}"),
           "max_err": float(e.max()), "p999_err": p999,
           "failing": int((e > PARITY_GATE).sum()), "pass": bool(ok),
           "oracle": ("FP64 raster with the BF16-emulating network (the GPU's network precision)" if bf16
                      else "FP64 raster and network"),
           "what": "max over the sampled unflagged pixels of |gpu - oracle| / max(1, |oracle|), per channel, "
                   "taken from the images of the last timed step", "oracle_seconds": t_par}
    if bf16:
        e64 = np.concatenate(e64_all)
        out["vs_fp64_network"] = {"max_err": float(e64.max()), "p999_err": float(np.quantile(e64, 0.999)),
                                  "mean_err": float(e64.mean())}
    return out


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
    # schedule: tile edge and per-block splat batch per scene, measured by the
    # library's autotuner (deferred path), or fixed by --tile / --batch
    scene_cfgs, tune = None, None
    tile_fixed = None if args.tile == "auto" else int(args.tile)
    if tile_fixed is None and (args.shading != "deferred" or args.vis_sh):
        tile_fixed = 16                 # the per-run schedule covers the fused deferred path only
    if tile_fixed is None:
        scene_cfgs, tune = PL.autotune_schedule(wl, precision=precision, reps=3)
    r = PL.renderer_for_workload(wl, precision=precision, tile=tile_fixed, batch=args.batch, vis_sh=vis_sh,
                                 shading=args.shading, scene_cfgs=scene_cfgs)
    n_inst = r.fit_capacity()
    schedule = None
    if scene_cfgs is not None:
        schedule = [{"scene": sc, "gaussians": wl.scenes[sc].N, "tile": c.tile, "batch": c.batch,
                     "candidates_ms": {f"{x.tile}x{x.tile}/{x.batch}": (round(x.ms, 4) if x.status == 0 else None)
                                       for x in tune[sc]}}
                    for sc, c in enumerate(scene_cfgs)]
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
    rt = PL.renderer_for_workload(wl_t, precision=precision)
    rt.fit_capacity()
    rt.forward()
    target = rt.img.clone()
    del rt
    torch.cuda.empty_cache()
    l1_scale = 1.0 / (3.0 * table.n_pixels)

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
            r.exchange_gradients()

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
    # pixels sampled from the timed batch's images for the parity check (the
    # oracle's values come from the CPU leg below)
    par_pix, par_got = {}, {}
    parity_ok = args.shading == "deferred" and not args.vis_sh
    if rank == 0 and world == 1 and not args.skip_cpu and parity_ok and args.parity_pixels > 0:
        import numpy as np
        rng = np.random.default_rng(2024)
        picks = sorted(set(np.linspace(0, n_pairs - 1, min(4, n_pairs)).round().astype(int).tolist()))
        for p in picks:
            pr = table.h[p]
            n_px = pr.W * pr.H
            sel = np.sort(rng.choice(n_px, min(args.parity_pixels, n_px), replace=False))
            par_pix[p] = np.stack([sel % pr.W, sel // pr.W], 1).astype(np.int32)
            idx = torch.from_numpy(pr.pixel_offset + sel).to("cuda")
            par_got[p] = r.img[idx].double().cpu().numpy()
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
    r.stats_fwd, r.stats_bwd = stats_f, stats_b
    for _ in range(reps if args.shading == "deferred" else 0):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(STAGES) + 1)]
        ev_v = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        if args.vis_sh:
            ev_v[0].record(st)
            B.vis_sh_fwd(table.h, table.d, r._scene_s, r.vis_sh, r.vis_item)
            ev_v[1].record(st)
        ev[0].record(st)
        r.run_stage("mlp_fwd")
        ev[1].record(st)
        r.run_stage("project_fwd")
        ev[2].record(st)
        r.run_stage("bin_sort")
        ev[3].record(st)
        r.run_stage("render_fwd")
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
            r.run_stage("render_bwd", dimg=r.dimg_loss)
            e_l[2].record(st)
            B.incident_loss(table.h, table.d, r.rec, 0.02, r.drec, r.loss)
            e_l[3].record(st)
        else:
            r.run_stage("render_bwd", target=target, l1_scale=l1_scale)
        ev[5].record(st)
        r.run_stage("mlp_bwd")
        ev[6].record(st)
        r.run_stage("project_bwd")
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
                "frac": ach / ALU_PEAK_TFLOPS, "traffic": kernel_traffic(dom, args.workload, n_pairs, (r.cfg.tile, r.cfg.batch) if r.groups is None
                                          else (0, 0)),
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
    # the metric's "% HBM roofline": compulsory bytes of the whole step (every
    # stage's algorithmic bytes) over the step time, against the measured peak
    hbm_roof = {"achieved": total_bytes / (ms_max * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                "frac": step_hbm_frac, "algorithmic_bytes_per_step": total_bytes, "target_frac": 0.5,
                "met": bool(step_hbm_frac >= 0.5), "peak_source": peak_src + " (hbm copy)",
                "what": "compulsory bytes of every stage of the step (projection, bin+sort, render forward and "
                        "backward, network, projection backward) per step time; the dominant kernel's own "
                        "fraction is roofline.hbm_frac_of_algorithmic_bytes"}

    # ---------------- the same step with the untuned schedule (16 x 16 tiles, 32-splat batches)
    untuned = None
    if schedule is not None and any((c["tile"], c["batch"]) != (16, 32) for c in schedule) and not args.no_graph:
        r0 = PL.renderer_for_workload(wl, precision=precision, tile=16, batch=32)
        r0.fit_capacity()
        g0 = r0.capture(target=target, l1_scale=l1_scale, loss=args.loss)
        for _ in range(max(args.warmup, 3)):
            g0.replay()
        torch.cuda.synchronize()
        u0 = torch.cuda.Event(enable_timing=True)
        u1 = torch.cuda.Event(enable_timing=True)
        u0.record(st)
        for _ in range(args.steps):
            g0.replay()
        u1.record(st)
        torch.cuda.synchronize()
        ums = u0.elapsed_time(u1) / args.steps
        untuned = {"renders_per_s": n_pairs * 1000.0 / ums, "ms_per_step": ums,
                   "what": "the same step with every scene on 16 x 16 tiles and 32-splat batches"}
        del r0, g0
        torch.cuda.empty_cache()

    # ---------------- unbatched per-pair paths: the plain FP32 baseline, and the
    # same with the tensor-core network, and with the fused kernels, which
    # split the batched path's speedup into network, fusion and batching
    plain = None
    speedup_split = None
    if not args.skip_plain:
        k = min(args.plain_pairs, n_pairs)
        reps_p = 3

        def per_pair(prec, fused):
            # one renderer per pair, each with buffers of its own pair's size
            rends = []
            for i in range(k):
                rp = PL.renderer_for_workload(wl, precision=prec, fused=fused, tile=16,
                                              pair_slice=slice(i, i + 1))
                rp.fit_capacity()
                rends.append((rp, torch.full((rp.table.n_pixels, 3), l1_scale, device="cuda")))

            def run():
                for rp, d in rends:
                    rp.forward()
                    rp.backward(dimg=d)
            run()
            torch.cuda.synchronize()
            rates = []
            for _ in range(reps_p):
                p0 = torch.cuda.Event(enable_timing=True)
                p1 = torch.cuda.Event(enable_timing=True)
                p0.record(st)
                run()
                p1.record(st)
                torch.cuda.synchronize()
                rates.append(k * 1000.0 / p0.elapsed_time(p1))
            del rends
            torch.cuda.empty_cache()
            return sorted(rates)[len(rates) // 2], rates

        pf, pf_all = per_pair(B.FP32, False)
        plain = {"renders_per_s": pf, "reps": pf_all, "pairs_timed": k,
                 "what": "per-pair launches, unfused composite and shade, FP32 CUDA-core network; median of "
                         f"{reps_p} repetitions over {k} pairs",
                 "speedup_of_batched": value / world / pf}
        if precision == B.BF16:
            pb, pb_all = per_pair(B.BF16, False)
            pu, pu_all = per_pair(B.BF16, True)
            speedup_split = {
                "plain_bf16_network_renders_per_s": pb, "per_pair_fused_renders_per_s": pu,
                "network": pb / pf, "fusion": pu / pb, "batching": value / world / pu,
                "what": ("plain FP32 -> tensor-core BF16 network (unfused, per pair) -> fused composite+shade "
                         "(per pair; these three on 16 x 16 tiles) -> one batched launch per stage over all pairs "
                         "under a CUDA graph, with the bench's schedule; the three factors multiply to "
                         "speedup_of_batched")}

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
                r.exchange_gradients()
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
                   "sample": (f"one pair of {args.workload}: network fwd+bwd over all {wl.scenes[wl.pairs[0].scene].N} Gaussians of its scene "
                              f"({d['t_mlp']:.1f} s) + raster fwd+bwd on every 16th pixel row "
                              f"({d['t_sample'] - d['t_mlp']:.1f} s) scaled by 16; single thread")}
        except Exception as ex:  # report, do not hide
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": f"failed: {ex}"[:300]}

    parity = None
    if par_pix:
        parity = parity_report(args, n_pairs, par_pix, par_got, precision == B.BF16)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "bf16+f32" if precision == B.BF16 else "f32",
                "data": "synthetic", "config": _config(args), "schedule": schedule, "untuned_schedule": untuned,
                "parity": parity,
                "roofline": roof, "hbm_roofline": hbm_roof, "step_hbm_frac_of_algorithmic": step_hbm_frac,
                "stage_ms": stage_ms, "loss_roofline": loss_roof, "visibility_trace": trace, "instances": n_inst, "items": n_items, "mlp_bwd_rows": n_active, "pixels": n_pixels,
                "contributions_per_step": {"forward": contrib_f, "backward": contrib_b},
                "cuda_graph": graph is not None,
                "plain_fp32": plain, "speedup_split": speedup_split, "e2e": e2e, "gpu_launches": int(launches), "clocks": clocks,
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
    c0 = B.launch_count()
    graph = r.capture(target=target, l1_scale=l1_scale)
    graph_launches = (B.launch_count() - c0) // 2

    def step():
        graph.replay()
        if world > 1:
            r.exchange_gradients()

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
                r.exchange_gradients()
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
    ap.add_argument("--tile", default="auto", choices=["auto", "8", "16", "32"],
                    help="tile edge; auto: per-scene tile edge and splat batch from the library's autotuner")
    ap.add_argument("--batch", type=int, default=None, choices=[None, 32, 64],
                    help="per-block splat batch of the render kernels with a fixed --tile (default 32)")
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
    ap.add_argument("--plain-pairs", type=int, default=8)
    ap.add_argument("--parity-pixels", type=int, default=1000,
                    help="pixels per sampled pair (4 pairs) compared with the oracle; 0 skips the check")
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
