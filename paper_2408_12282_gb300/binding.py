"""ctypes binding of libsssgs (include/sssgs.h): argument marshalling only.

Every function here has the name of the C entry point without the `sssgs_`
prefix, takes torch tensors (or None) for device pointers, and raises
SSSGSError on a non-zero return code. No compute happens in Python.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

c_i32, c_i64, c_f32, c_vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_void_p
MAX_LAYERS = 8
NF, REC, GBUF, DX = 15, 24, 16, 14
MLP_BASIC, MLP_PE6, MLP_PAPER = 0, 1, 2
FP32, BF16 = 0, 1
STATUS_CAPACITY = 1
STATUS_TIMEOUT = 2


class SSSGSError(RuntimeError):
    pass


class Cfg(ctypes.Structure):
    _fields_ = [("tile", c_i32), ("batch", c_i32), ("dilation", c_f32), ("det_eps", c_f32),
                ("z_near", c_f32), ("alpha_min", c_f32), ("alpha_max", c_f32), ("T_min", c_f32),
                ("A_eps", c_f32)]


class Pair(ctypes.Structure):
    _fields_ = [("R", c_f32 * 9), ("t", c_f32 * 3), ("fx", c_f32), ("fy", c_f32), ("cx", c_f32),
                ("cy", c_f32), ("light", c_f32 * 3), ("W", c_i32), ("H", c_i32), ("g_begin", c_i32),
                ("g_count", c_i32), ("tiles_x", c_i32), ("tiles_y", c_i32), ("tile_offset", c_i32),
                ("pad0", c_i32), ("pad1", c_i32), ("pixel_offset", c_i64), ("item_offset", c_i64)]


assert ctypes.sizeof(Pair) == 128


class PlanInfo(ctypes.Structure):
    _fields_ = [("n_items", c_i64), ("n_pixels", c_i64), ("n_tiles", c_i32), ("tile_bits", c_i32)]


_SCENE_FIELDS = ("mu", "log_s", "quat", "logit_o", "normal", "base", "rough", "metal", "sss", "vis")


class Scene(ctypes.Structure):
    _fields_ = [(k, c_vp) for k in _SCENE_FIELDS] + [("n", c_i64), ("vis_item", c_vp)]


class SceneGrad(ctypes.Structure):
    _fields_ = [(k, c_vp) for k in _SCENE_FIELDS] + [("vis_item", c_vp)]


class MLP(ctypes.Structure):
    _fields_ = [("kind", c_i32), ("n_layers", c_i32), ("precision", c_i32),
                ("width", c_i32 * (MAX_LAYERS + 1)), ("W", c_vp * MAX_LAYERS), ("b", c_vp * MAX_LAYERS)]


class MLPGrad(ctypes.Structure):
    _fields_ = [("W", c_vp * MAX_LAYERS), ("b", c_vp * MAX_LAYERS)]


class TuneBuffers(ctypes.Structure):
    _fields_ = [("d_pairs", c_vp), ("rec", c_vp), ("rect", c_vp), ("vals", c_vp), ("capacity", c_i64),
                ("ranges", c_vp), ("max_tiles", c_i32), ("pad", c_i32), ("d_count", c_vp), ("d_status", c_vp),
                ("workspace", c_vp), ("workspace_bytes", ctypes.c_size_t), ("gbuf", c_vp), ("last", c_vp),
                ("img", c_vp), ("drec", c_vp), ("dimg", c_vp)]


class TuneResult(ctypes.Structure):
    _fields_ = [("tile", c_i32), ("batch", c_i32), ("status", c_i32), ("reps", c_i32), ("instances", c_i64),
                ("ms", c_f32), ("reserved", c_f32)]


assert ctypes.sizeof(TuneResult) == 32


_LIB = None

_SIGS = {
    "sssgs_version": ([], ctypes.c_char_p),
    "sssgs_launch_count": ([], ctypes.c_uint64),
    "sssgs_strerror": ([ctypes.c_int], ctypes.c_char_p),
    "sssgs_cfg_default": ([ctypes.POINTER(Cfg)], None),
    "sssgs_plan": ([ctypes.POINTER(Pair), ctypes.c_int, ctypes.POINTER(Cfg), ctypes.POINTER(PlanInfo)], ctypes.c_int),
    "sssgs_mlp_fwd": ([ctypes.POINTER(MLP), ctypes.POINTER(Pair), c_vp, ctypes.c_int, ctypes.POINTER(Scene), c_vp,
                       c_vp, c_vp], ctypes.c_int),
    "sssgs_mlp_workspace_bytes": ([ctypes.POINTER(MLP), c_i64], ctypes.c_size_t),
    "sssgs_mlp_bwd": ([ctypes.POINTER(MLP), ctypes.POINTER(Pair), c_vp, ctypes.c_int, ctypes.POINTER(Scene), c_vp,
                       ctypes.POINTER(MLPGrad), c_vp, c_vp, ctypes.c_size_t, c_vp, c_vp], ctypes.c_int),
    "sssgs_mlp_bwd_strided": ([ctypes.POINTER(MLP), ctypes.POINTER(Pair), c_vp, ctypes.c_int,
                               ctypes.POINTER(Scene), c_vp, c_i64, ctypes.POINTER(MLPGrad), c_vp, c_vp,
                               ctypes.c_size_t, c_vp, c_vp], ctypes.c_int),
    "sssgs_project_fwd": ([ctypes.POINTER(Cfg), ctypes.POINTER(Pair), c_vp, ctypes.c_int, ctypes.POINTER(Scene),
                           c_vp, c_vp, c_vp, c_vp], ctypes.c_int),
    "sssgs_bin_workspace_bytes": ([c_i64, c_i64, c_i32], ctypes.c_size_t),
    "sssgs_bin_sort": ([ctypes.POINTER(Cfg), ctypes.POINTER(Pair), c_vp, ctypes.c_int, c_vp, c_vp, c_i64, c_vp,
                        c_vp, c_vp, c_vp, c_vp, ctypes.c_size_t, c_vp], ctypes.c_int),
    "sssgs_bin_sort_static": ([ctypes.POINTER(Cfg), ctypes.POINTER(Pair), c_vp, ctypes.c_int, c_vp, c_vp, c_i64,
                               c_vp, c_vp, c_vp, c_vp, c_vp], ctypes.c_int),
    "sssgs_composite_fwd": ([ctypes.POINTER(Cfg), ctypes.POINTER(Pair), c_vp, ctypes.c_int, c_vp, c_vp, c_vp, c_vp,
                             c_vp, c_vp], ctypes.c_int),
    "sssgs_shade_fwd": ([ctypes.POINTER(Cfg), ctypes.POINTER(Pair), c_vp, ctypes.c_int, c_vp, c_vp, c_vp],
                        ctypes.c_int),
    "sssgs_shade_bwd": ([ctypes.POINTER(Cfg), ctypes.POINTER(Pair), c_vp, ctypes.c_int, c_vp, c_vp, c_vp, c_vp],
                        ctypes.c_int),
    "sssgs_composite_bwd": ([ctypes.POINTER(Cfg), ctypes.POINTER(Pair), c_vp, ctypes.c_int, c_vp, c_vp, c_vp, c_vp,
                             c_vp, c_vp, c_vp, c_vp], ctypes.c_int),
    "sssgs_render_fwd": ([ctypes.POINTER(Cfg), ctypes.POINTER(Pair), c_vp, ctypes.c_int, c_vp, c_vp, c_vp, c_vp,
                          c_vp, c_vp, c_vp, c_vp], ctypes.c_int),
    "sssgs_render_bwd": ([ctypes.POINTER(Cfg), ctypes.POINTER(Pair), c_vp, ctypes.c_int, c_vp, c_vp, c_vp, c_vp,
                          c_vp, c_vp, c_vp, c_vp, c_vp, c_f32, c_vp, c_vp, c_vp], ctypes.c_int),
    "sssgs_autotune": ([ctypes.POINTER(Cfg), ctypes.POINTER(Pair), ctypes.c_int, ctypes.POINTER(Scene), c_vp,
                        ctypes.POINTER(TuneBuffers), ctypes.POINTER(c_i32), ctypes.c_int, ctypes.POINTER(c_i32),
                        ctypes.c_int, ctypes.c_int, ctypes.POINTER(TuneResult), ctypes.POINTER(Cfg), c_vp],
                       ctypes.c_int),
    "sssgs_project_bwd": ([ctypes.POINTER(Cfg), ctypes.POINTER(Pair), c_vp, ctypes.c_int, ctypes.POINTER(Scene),
                           c_vp, c_vp, ctypes.POINTER(SceneGrad), c_vp], ctypes.c_int),
    "sssgs_render_ml_fwd": ([ctypes.POINTER(Cfg), ctypes.POINTER(Pair), c_vp, ctypes.c_int, ctypes.c_int, c_vp,
                             c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp], ctypes.c_int),
    "sssgs_render_ml_bwd": ([ctypes.POINTER(Cfg), ctypes.POINTER(Pair), c_vp, ctypes.c_int, ctypes.c_int, c_vp,
                             c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_f32, c_vp, c_vp, c_vp, c_vp],
                            ctypes.c_int),
    "sssgs_bvh_floats": ([c_i64], c_i64),
    "sssgs_bvh_workspace_bytes": ([c_i64], ctypes.c_size_t),
    "sssgs_bvh_build": ([ctypes.POINTER(Cfg), ctypes.POINTER(Scene), c_vp, c_vp, ctypes.c_size_t, c_vp], ctypes.c_int),
    "sssgs_trace_visibility": ([ctypes.POINTER(Cfg), ctypes.POINTER(Pair), c_vp, ctypes.c_int, ctypes.POINTER(Scene),
                                c_vp, c_vp, c_vp], ctypes.c_int),
    "sssgs_vis_sh_fwd": ([ctypes.POINTER(Pair), c_vp, ctypes.c_int, ctypes.POINTER(Scene), c_vp, c_vp, c_vp],
                         ctypes.c_int),
    "sssgs_vis_sh_bwd": ([ctypes.POINTER(Pair), c_vp, ctypes.c_int, ctypes.POINTER(Scene), c_vp, c_vp, c_vp, c_vp,
                          c_vp], ctypes.c_int),
    "sssgs_vis_loss": ([ctypes.POINTER(Pair), c_vp, ctypes.c_int, c_vp, c_vp, c_f32, c_vp, c_vp, c_vp], ctypes.c_int),
    "sssgs_selftest_wait_timeout": ([c_vp, c_i64, c_vp], ctypes.c_int),
    "sssgs_shade_gaussians_fwd": ([ctypes.POINTER(Pair), c_vp, ctypes.c_int, ctypes.POINTER(Scene), c_vp, c_vp,
                                   c_vp], ctypes.c_int),
    "sssgs_shade_gaussians_bwd": ([ctypes.POINTER(Pair), c_vp, ctypes.c_int, ctypes.POINTER(Scene), c_vp, c_vp,
                                   c_vp], ctypes.c_int),
    "sssgs_colors_to_image": ([ctypes.POINTER(Pair), ctypes.c_int, c_vp, c_vp, c_vp], ctypes.c_int),
    "sssgs_colors_to_image_bwd": ([ctypes.POINTER(Pair), ctypes.c_int, c_vp, c_vp, c_vp], ctypes.c_int),
    "sssgs_image_loss_workspace_bytes": ([c_i64], ctypes.c_size_t),
    "sssgs_image_loss": ([ctypes.POINTER(Cfg), ctypes.POINTER(Pair), c_vp, ctypes.c_int, c_vp, c_vp, c_f32, c_vp,
                          c_vp, c_vp, ctypes.c_size_t, c_vp], ctypes.c_int),
    "sssgs_incident_loss": ([ctypes.POINTER(Pair), c_vp, ctypes.c_int, c_vp, c_f32, c_vp, c_vp, c_vp], ctypes.c_int),
}

EXPORTED = tuple(_SIGS)


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True):
    """Load libsssgs.so; raise if it is missing (there is no fallback path)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise SSSGSError(f"CUDA library not built: {path}")
        _build.build()
    lib = ctypes.CDLL(path)
    for name, (args, res) in _SIGS.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _LIB = lib
    return lib


def _p(t):
    """Device (or host) address of a tensor argument. Every buffer of the C ABI
    is float32, int32/uint32, uint8 or int64 and dense: a float64 or strided
    tensor would be read with the wrong layout, so it is refused here."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if t.dtype == torch.float64 or t.dtype == torch.float16 or t.dtype == torch.bfloat16:
        raise TypeError(f"sssgs buffers are float32; got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError("sssgs buffers must be contiguous")
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _check(rc, name):
    if rc != 0:
        msg = load_library().sssgs_strerror(rc).decode()
        raise SSSGSError(f"{name} failed: {rc} ({msg})")


# --------------------------------------------------------------------------- structs

def cfg_default() -> Cfg:
    c = Cfg()
    load_library().sssgs_cfg_default(ctypes.byref(c))
    return c


def version() -> str:
    return load_library().sssgs_version().decode()


def launch_count() -> int:
    return int(load_library().sssgs_launch_count())


def strerror(code: int) -> str:
    return load_library().sssgs_strerror(code).decode()


def plan(pairs_arr, cfg: Cfg) -> PlanInfo:
    info = PlanInfo()
    _check(load_library().sssgs_plan(pairs_arr, len(pairs_arr), ctypes.byref(cfg), ctypes.byref(info)), "sssgs_plan")
    return info


def scene_struct(t: dict, vis_item=None) -> Scene:
    """vis_item: optional per-item visibility (n_items floats)."""
    return Scene(*[_p(t[k]) for k in _SCENE_FIELDS], t["mu"].shape[0], _p(vis_item))


def scene_grad_struct(t: dict, vis_item=None) -> SceneGrad:
    return SceneGrad(*[_p(t.get(k)) for k in _SCENE_FIELDS], _p(vis_item))


def mlp_struct(kind: int, precision: int, Ws, bs) -> MLP:
    m = MLP()
    m.kind = kind
    m.precision = precision
    m.n_layers = len(Ws)
    m.width[0] = Ws[0].shape[1]
    for l, W in enumerate(Ws):
        m.width[l + 1] = W.shape[0]
        m.W[l] = _p(W)
        m.b[l] = _p(bs[l])
    return m


def mlp_grad_struct(dWs, dbs) -> MLPGrad:
    g = MLPGrad()
    for l, W in enumerate(dWs):
        g.W[l] = _p(W)
        g.b[l] = _p(dbs[l]) if dbs is not None else None
    return g


# --------------------------------------------------------------------------- entry points

def mlp_fwd(mlp: MLP, pairs, d_pairs, scene: Scene, out, d_status=None, stream=None):
    _check(load_library().sssgs_mlp_fwd(ctypes.byref(mlp), pairs, _p(d_pairs), len(pairs), ctypes.byref(scene),
                                        _p(out), _p(d_status), _stream(stream)), "sssgs_mlp_fwd")


def mlp_workspace_bytes(mlp: MLP, n_items: int) -> int:
    return int(load_library().sssgs_mlp_workspace_bytes(ctypes.byref(mlp), n_items))


def mlp_bwd(mlp: MLP, pairs, d_pairs, scene: Scene, drec, grad: MLPGrad, dx_items, workspace, d_status=None,
            stream=None):
    _check(load_library().sssgs_mlp_bwd(ctypes.byref(mlp), pairs, _p(d_pairs), len(pairs), ctypes.byref(scene),
                                        _p(drec), ctypes.byref(grad), _p(dx_items), _p(workspace),
                                        workspace.numel() * workspace.element_size() if workspace is not None else 0,
                                        _p(d_status), _stream(stream)), "sssgs_mlp_bwd")


def project_fwd(cfg: Cfg, pairs, d_pairs, scene: Scene, mlp_out, rec, rect, stream=None):
    _check(load_library().sssgs_project_fwd(ctypes.byref(cfg), pairs, _p(d_pairs), len(pairs), ctypes.byref(scene),
                                            _p(mlp_out), _p(rec), _p(rect), _stream(stream)), "sssgs_project_fwd")


def bin_workspace_bytes(n_items: int, capacity: int, n_tiles: int) -> int:
    return int(load_library().sssgs_bin_workspace_bytes(n_items, capacity, n_tiles))


def bin_sort(cfg: Cfg, pairs, d_pairs, rec, rect, capacity: int, vals, ranges, d_count, d_status, workspace,
             stream=None):
    _check(load_library().sssgs_bin_sort(ctypes.byref(cfg), pairs, _p(d_pairs), len(pairs), _p(rec), _p(rect),
                                         capacity, _p(vals), _p(ranges), _p(d_count), _p(d_status), _p(workspace),
                                         workspace.numel() * workspace.element_size(), _stream(stream)),
           "sssgs_bin_sort")


STATIC_MAX_ITEMS = 65536
STATIC_MAX_INSTANCES = 524288
ERR_INVALID_ARG = -1
ERR_WORKSPACE = -4
ERR_TOO_LARGE = -5


def bin_sort_static(cfg: Cfg, pairs, d_pairs, rec, rect, capacity: int, vals, ranges, d_count, d_status,
                    stream=None):
    """bin_sort without a workspace: for callers that cannot allocate device
    memory; runs in the library's fixed scratch (limits above)."""
    _check(load_library().sssgs_bin_sort_static(ctypes.byref(cfg), pairs, _p(d_pairs), len(pairs), _p(rec),
                                                _p(rect), capacity, _p(vals), _p(ranges), _p(d_count),
                                                _p(d_status), _stream(stream)), "sssgs_bin_sort_static")


def composite_fwd(cfg: Cfg, pairs, d_pairs, rec, vals, ranges, gbuf, last, stream=None):
    _check(load_library().sssgs_composite_fwd(ctypes.byref(cfg), pairs, _p(d_pairs), len(pairs), _p(rec), _p(vals),
                                              _p(ranges), _p(gbuf), _p(last), _stream(stream)),
           "sssgs_composite_fwd")


def shade_fwd(cfg: Cfg, pairs, d_pairs, gbuf, img, stream=None):
    _check(load_library().sssgs_shade_fwd(ctypes.byref(cfg), pairs, _p(d_pairs), len(pairs), _p(gbuf), _p(img),
                                          _stream(stream)), "sssgs_shade_fwd")


def shade_bwd(cfg: Cfg, pairs, d_pairs, gbuf, dimg, dgbuf, stream=None):
    _check(load_library().sssgs_shade_bwd(ctypes.byref(cfg), pairs, _p(d_pairs), len(pairs), _p(gbuf), _p(dimg),
                                          _p(dgbuf), _stream(stream)), "sssgs_shade_bwd")


def composite_bwd(cfg: Cfg, pairs, d_pairs, rec, vals, ranges, gbuf, last, dgbuf, drec, stream=None):
    _check(load_library().sssgs_composite_bwd(ctypes.byref(cfg), pairs, _p(d_pairs), len(pairs), _p(rec), _p(vals),
                                              _p(ranges), _p(gbuf), _p(last), _p(dgbuf), _p(drec),
                                              _stream(stream)), "sssgs_composite_bwd")


def render_fwd(cfg: Cfg, pairs, d_pairs, rec, vals, ranges, gbuf, last, img, stats=None, stream=None):
    _check(load_library().sssgs_render_fwd(ctypes.byref(cfg), pairs, _p(d_pairs), len(pairs), _p(rec), _p(vals),
                                           _p(ranges), _p(gbuf), _p(last), _p(img), _p(stats), _stream(stream)),
           "sssgs_render_fwd")


def render_bwd(cfg: Cfg, pairs, d_pairs, rec, vals, ranges, gbuf, last, img, dimg, target, weight, l1_scale,
               drec, stats=None, stream=None):
    _check(load_library().sssgs_render_bwd(ctypes.byref(cfg), pairs, _p(d_pairs), len(pairs), _p(rec), _p(vals),
                                           _p(ranges), _p(gbuf), _p(last), _p(img), _p(dimg), _p(target),
                                           _p(weight), float(l1_scale), _p(drec), _p(stats), _stream(stream)),
           "sssgs_render_bwd")


def autotune(base: Cfg, pairs, scene: Scene, mlp_out, buffers: TuneBuffers, tiles, batches, reps: int,
             stream=None):
    """Time every (tile, batch) candidate of the schedule-dependent stages on
    one scene's pairs (sssgs_autotune). Returns (best Cfg, list of
    TuneResult); best is None when no candidate's instances fitted the
    buffers' capacity (each result then holds its instance count). Blocking;
    call outside stream capture."""
    tl = (c_i32 * len(tiles))(*[int(t) for t in tiles])
    bl = (c_i32 * len(batches))(*[int(b) for b in batches])
    res = (TuneResult * (len(tiles) * len(batches)))()
    best = Cfg()
    rc = load_library().sssgs_autotune(ctypes.byref(base), pairs, len(pairs), ctypes.byref(scene), _p(mlp_out),
                                       ctypes.byref(buffers), tl, len(tiles), bl, len(batches), int(reps), res,
                                       ctypes.byref(best), _stream(stream))
    if rc == ERR_WORKSPACE and all(r.status == STATUS_CAPACITY for r in res):
        return None, list(res)       # no candidate fitted the capacity: results hold the instance counts
    _check(rc, "sssgs_autotune")
    return best, list(res)


def mlp_bwd_strided(mlp: MLP, pairs, d_pairs, scene: Scene, dout, dout_stride: int, grad: MLPGrad, dx_items,
                    workspace, d_status=None, stream=None):
    _check(load_library().sssgs_mlp_bwd_strided(ctypes.byref(mlp), pairs, _p(d_pairs), len(pairs),
                                                ctypes.byref(scene), _p(dout), int(dout_stride), ctypes.byref(grad),
                                                _p(dx_items), _p(workspace),
                                                workspace.numel() * workspace.element_size()
                                                if workspace is not None else 0, _p(d_status), _stream(stream)),
           "sssgs_mlp_bwd_strided")


def render_ml_fwd(cfg: Cfg, views, d_views, n_lights: int, lights, rec, mlp_out, vals, ranges, gbuf, last, img,
                  env_w=None, stats=None, stream=None):
    _check(load_library().sssgs_render_ml_fwd(ctypes.byref(cfg), views, _p(d_views), len(views), int(n_lights),
                                              _p(lights), _p(rec), _p(mlp_out), _p(vals), _p(ranges), _p(gbuf),
                                              _p(last), _p(img), _p(env_w), _p(stats), _stream(stream)),
           "sssgs_render_ml_fwd")


def render_ml_bwd(cfg: Cfg, views, d_views, n_lights: int, lights, rec, mlp_out, vals, ranges, gbuf, last, img,
                  dimg, target, l1_scale, drec, dmlp, stats=None, stream=None):
    _check(load_library().sssgs_render_ml_bwd(ctypes.byref(cfg), views, _p(d_views), len(views), int(n_lights),
                                              _p(lights), _p(rec), _p(mlp_out), _p(vals), _p(ranges), _p(gbuf),
                                              _p(last), _p(img), _p(dimg), _p(target), float(l1_scale), _p(drec),
                                              _p(dmlp), _p(stats), _stream(stream)),
           "sssgs_render_ml_bwd")


def project_bwd(cfg: Cfg, pairs, d_pairs, scene: Scene, drec, dx_items, grad: SceneGrad, stream=None):
    _check(load_library().sssgs_project_bwd(ctypes.byref(cfg), pairs, _p(d_pairs), len(pairs), ctypes.byref(scene),
                                            _p(drec), _p(dx_items), ctypes.byref(grad), _stream(stream)),
           "sssgs_project_bwd")


def selftest_wait_timeout(d_status, limit_cycles: int, stream=None):
    _check(load_library().sssgs_selftest_wait_timeout(_p(d_status), int(limit_cycles), _stream(stream)),
           "sssgs_selftest_wait_timeout")


def shade_gaussians_fwd(pairs, d_pairs, scene: Scene, rec, rec_colors, stream=None):
    _check(load_library().sssgs_shade_gaussians_fwd(pairs, _p(d_pairs), len(pairs), ctypes.byref(scene), _p(rec),
                                                    _p(rec_colors), _stream(stream)), "sssgs_shade_gaussians_fwd")


def shade_gaussians_bwd(pairs, d_pairs, scene: Scene, rec, drec, stream=None):
    _check(load_library().sssgs_shade_gaussians_bwd(pairs, _p(d_pairs), len(pairs), ctypes.byref(scene), _p(rec),
                                                    _p(drec), _stream(stream)), "sssgs_shade_gaussians_bwd")


def colors_to_image(pairs, gbuf, img, stream=None):
    _check(load_library().sssgs_colors_to_image(pairs, len(pairs), _p(gbuf), _p(img), _stream(stream)),
           "sssgs_colors_to_image")


def colors_to_image_bwd(pairs, dimg, dgbuf, stream=None):
    _check(load_library().sssgs_colors_to_image_bwd(pairs, len(pairs), _p(dimg), _p(dgbuf), _stream(stream)),
           "sssgs_colors_to_image_bwd")


def bvh_floats(n: int) -> int:
    return int(load_library().sssgs_bvh_floats(n))


def bvh_workspace_bytes(n: int) -> int:
    return int(load_library().sssgs_bvh_workspace_bytes(n))


def bvh_build(cfg: Cfg, scene: Scene, bvh, workspace, stream=None):
    _check(load_library().sssgs_bvh_build(ctypes.byref(cfg), ctypes.byref(scene), _p(bvh), _p(workspace),
                                          workspace.numel() * workspace.element_size(), _stream(stream)),
           "sssgs_bvh_build")


def trace_visibility(cfg: Cfg, pairs, d_pairs, scene: Scene, bvh, vis_traced, stream=None):
    _check(load_library().sssgs_trace_visibility(ctypes.byref(cfg), pairs, _p(d_pairs), len(pairs),
                                                 ctypes.byref(scene), _p(bvh), _p(vis_traced), _stream(stream)),
           "sssgs_trace_visibility")


def vis_sh_fwd(pairs, d_pairs, scene: Scene, vis_sh, vis_item, stream=None):
    _check(load_library().sssgs_vis_sh_fwd(pairs, _p(d_pairs), len(pairs), ctypes.byref(scene), _p(vis_sh),
                                           _p(vis_item), _stream(stream)), "sssgs_vis_sh_fwd")


def vis_sh_bwd(pairs, d_pairs, scene: Scene, vis_sh, dvis_item, dvis_sh, dmu, stream=None):
    _check(load_library().sssgs_vis_sh_bwd(pairs, _p(d_pairs), len(pairs), ctypes.byref(scene), _p(vis_sh),
                                           _p(dvis_item), _p(dvis_sh), _p(dmu), _stream(stream)), "sssgs_vis_sh_bwd")


def vis_loss(pairs, d_pairs, vis_item, vis_traced, lambda_raytrace, dvis_item, d_loss, stream=None):
    _check(load_library().sssgs_vis_loss(pairs, _p(d_pairs), len(pairs), _p(vis_item), _p(vis_traced),
                                         float(lambda_raytrace), _p(dvis_item), _p(d_loss), _stream(stream)),
           "sssgs_vis_loss")


def image_loss_workspace_bytes(n_pixels: int) -> int:
    return int(load_library().sssgs_image_loss_workspace_bytes(n_pixels))


def image_loss(cfg: Cfg, pairs, d_pairs, img, target, lambda_dssim, dimg, d_loss, workspace, stream=None):
    _check(load_library().sssgs_image_loss(ctypes.byref(cfg), pairs, _p(d_pairs), len(pairs), _p(img), _p(target),
                                           float(lambda_dssim), _p(dimg), _p(d_loss), _p(workspace),
                                           workspace.numel() * workspace.element_size(), _stream(stream)),
           "sssgs_image_loss")


def incident_loss(pairs, d_pairs, rec, lambda_incident, drec, d_loss, stream=None):
    _check(load_library().sssgs_incident_loss(pairs, _p(d_pairs), len(pairs), _p(rec), float(lambda_incident),
                                              _p(drec), _p(d_loss), _stream(stream)), "sssgs_incident_loss")
