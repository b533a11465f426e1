"""The C-ABI library loads and exports every entry point include/sssgs.h
declares; host-only entry points behave (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest
import torch

from paper_2408_12282_gb300 import binding as B

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "sssgs.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sssgs_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported():
    lib = B.load_library()
    names = _declared()
    assert len(names) >= 17
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding covers every one of them under the same name
    assert set(names) <= set(B.EXPORTED), set(names) - set(B.EXPORTED)


def test_struct_layouts_match_header():
    assert ctypes.sizeof(B.Pair) == 128
    assert ctypes.sizeof(B.Cfg) == 36
    assert ctypes.sizeof(B.MLP) == 4 * 3 + 4 * 9 + 8 * 16
    assert B.Pair.pixel_offset.offset == 112 and B.Pair.item_offset.offset == 120
    assert ctypes.sizeof(B.TuneBuffers) == 128 and B.TuneBuffers.workspace_bytes.offset == 80
    assert ctypes.sizeof(B.TuneResult) == 32 and B.TuneResult.ms.offset == 24


def test_autotune_rejects_bad_arguments_before_any_launch():
    """Host-side checks of sssgs_autotune (no GPU needed): missing buffers,
    reps out of range, a batch other than 32 or 64, an empty candidate list."""
    lib = B.load_library()
    base = B.cfg_default()
    h = (B.Pair * 1)()
    h[0].W, h[0].H, h[0].fx, h[0].fy, h[0].g_count = 64, 64, 50.0, 50.0, 10
    scene = B.Scene()
    tiles = (ctypes.c_int32 * 2)(8, 16)
    batches = (ctypes.c_int32 * 1)(32)
    res = (B.TuneResult * 2)()
    best = B.Cfg()
    empty = B.TuneBuffers()
    rc = lib.sssgs_autotune(ctypes.byref(base), h, 1, ctypes.byref(scene), 16, ctypes.byref(empty), tiles, 2, batches,
                            1, 3, res, ctypes.byref(best), None)
    assert rc == B.ERR_INVALID_ARG
    full = B.TuneBuffers()
    for k in ("d_pairs", "rec", "rect", "vals", "ranges", "d_count", "d_status", "gbuf", "last", "img", "drec",
              "dimg"):
        setattr(full, k, 256)
    for reps, bt in ((0, 32), (1001, 32), (3, 48)):
        batches[0] = bt
        rc = lib.sssgs_autotune(ctypes.byref(base), h, 1, ctypes.byref(scene), 16, ctypes.byref(full), tiles, 2,
                                batches, 1, reps, res, ctypes.byref(best), None)
        assert rc == B.ERR_INVALID_ARG, (reps, bt)
    batches[0] = 32
    rc = lib.sssgs_autotune(ctypes.byref(base), h, 1, ctypes.byref(scene), 16, ctypes.byref(full), tiles, 0,
                            batches, 1, 3, res, ctypes.byref(best), None)
    assert rc == B.ERR_INVALID_ARG
    full.max_tiles = 10            # 8 x 8 tiles of a 64 x 64 image need 64
    rc = lib.sssgs_autotune(ctypes.byref(base), h, 1, ctypes.byref(scene), 16, ctypes.byref(full), tiles, 2,
                            batches, 1, 3, res, ctypes.byref(best), None)
    assert rc == B.ERR_INVALID_ARG


def test_defaults_and_strerror():
    c = B.cfg_default()
    assert c.tile == 16 and c.batch == 32
    assert c.alpha_min == pytest.approx(np.float32(1 / 255))
    assert c.alpha_max == pytest.approx(np.float32(0.99))
    assert c.T_min == pytest.approx(np.float32(1e-4))
    assert B.strerror(0) == "ok"
    assert "invalid" in B.strerror(-1)
    assert B.version().startswith("sssgs")


def test_plan_offsets_and_validation():
    c = B.cfg_default()
    sizes = [(800, 800), (400, 400), (1600, 1200), (7, 5)]
    h = (B.Pair * len(sizes))()
    for k, (w, hh) in enumerate(sizes):
        h[k].W, h[k].H, h[k].fx, h[k].fy = w, hh, 100.0, 100.0
        h[k].g_begin, h[k].g_count = 10 * k, 1000 + k
    info = B.plan(h, c)
    tiles = [((w + 15) // 16) * ((hh + 15) // 16) for w, hh in sizes]
    assert info.n_tiles == sum(tiles)
    assert info.n_pixels == sum(w * hh for w, hh in sizes)
    assert info.n_items == sum(1000 + k for k in range(4))
    assert [h[k].tile_offset for k in range(4)] == list(np.cumsum([0] + tiles[:-1]))
    assert [h[k].item_offset for k in range(4)] == [0, 1000, 2001, 3003]
    assert (1 << info.tile_bits) >= info.n_tiles > (1 << (info.tile_bits - 1))
    h[1].W = 0
    with pytest.raises(B.SSSGSError):
        B.plan(h, c)
    c.tile = 12
    h[1].W = 400
    with pytest.raises(B.SSSGSError):
        B.plan(h, c)


def test_workspace_queries():
    assert B.bin_workspace_bytes(0, 0, 1) > 0
    a = B.bin_workspace_bytes(1000, 10000, 100)
    b = B.bin_workspace_bytes(1000, 20000, 100)
    assert b > a >= 1000 * 32 + 10000 * 12


def test_argument_errors_launch_nothing():
    """Host-side checks reject bad arguments before touching the device."""
    lib = B.load_library()
    c = B.cfg_default()
    h = (B.Pair * 1)()
    h[0].W = h[0].H = 16
    h[0].fx = h[0].fy = 10.0
    B.plan(h, c)
    assert lib.sssgs_project_fwd(ctypes.byref(c), h, None, 1, None, None, None, None, None) == -1
    assert lib.sssgs_composite_fwd(ctypes.byref(c), h, None, 1, None, None, None, None, None, None) == -1
    c.tile = 5
    assert lib.sssgs_render_fwd(ctypes.byref(c), h, 16, 1, 16, 16, 16, 16, 16, 16, None, None) == -1
    assert lib.sssgs_bin_sort(ctypes.byref(c), h, 16, 1, 16, 16, -1, 16, 16, 16, 16, 16, 0, None) == -1


def test_binding_refuses_float64_and_strided_buffers():
    """Every buffer of the C ABI is dense float32 / int32 / uint8 / int64: a
    float64 or strided tensor would be read with the wrong layout, so the
    binding refuses it before any call."""
    with pytest.raises(TypeError):
        B._p(torch.zeros(4, 3, dtype=torch.float64))
    with pytest.raises(ValueError):
        B._p(torch.zeros(4, 6)[:, ::2])
    assert B._p(None) is None
    assert B._p(torch.zeros(4, 3)) != 0


def test_later_entry_points_reject_bad_arguments():
    """The many-light, visibility, loss and per-Gaussian shading entry points
    check their host arguments before any device work: a missing buffer, an
    unsupported light count or tile edge, a misaligned buffer or a loss
    weight outside [0, 1] returns an error code (fake aligned addresses
    stand in for device buffers; nothing is dereferenced or launched)."""
    lib = B.load_library()
    c = B.cfg_default()
    h = (B.Pair * 1)()
    h[0].W = h[0].H = 16
    h[0].fx = h[0].fy = 10.0
    B.plan(h, c)
    A = 256                      # an aligned fake device address
    INVALID, UNSUPPORTED = -1, -3
    ml = lambda cfg, d, L, rec: lib.sssgs_render_ml_fwd(ctypes.byref(cfg), h, d, 1, L, A, rec, A, A, A, A, A, A,
                                                        None, None, None)
    assert ml(c, None, 8, A) == INVALID                   # no device pair table
    assert ml(c, A, 3, A) == INVALID                      # light count not 1, 2, 4, 8
    assert ml(c, A, 8, A + 4) == INVALID                  # records not 16-byte aligned
    c8 = B.cfg_default()
    c8.tile = 8
    assert ml(c8, A, 8, A) == UNSUPPORTED                 # many-light kernels are 16 x 16 only
    assert lib.sssgs_render_ml_bwd(ctypes.byref(c), h, A, 1, 8, A, A, A, A, A, A, A, None, None, None, 1.0,
                                   A, A, None, None) == INVALID   # neither dimg nor (img, target)
    sc = B.Scene()
    assert lib.sssgs_bvh_build(ctypes.byref(c), ctypes.byref(sc), A, A, 0, None) == INVALID   # no scene arrays
    assert lib.sssgs_trace_visibility(ctypes.byref(c), h, A, 1, ctypes.byref(sc), A, A, None) == INVALID
    assert lib.sssgs_vis_sh_fwd(h, A, 1, ctypes.byref(sc), A, A, None) == INVALID
    assert lib.sssgs_vis_loss(h, A, 1, A, None, 0.01, A, A, None) == INVALID
    assert lib.sssgs_image_loss(ctypes.byref(c), h, A, 1, A, A, 1.5, A, A, A, 1 << 20, None) == INVALID
    assert lib.sssgs_image_loss(ctypes.byref(c), h, A, 1, A, None, 0.2, A, A, A, 1 << 20, None) == INVALID
    assert lib.sssgs_incident_loss(h, A, 1, None, 0.02, A, A, None) == INVALID
    assert lib.sssgs_shade_gaussians_fwd(h, A, 1, ctypes.byref(sc), A, A, None) == INVALID
    assert lib.sssgs_colors_to_image(h, 1, A + 4, A, None) == INVALID   # G-buffer not 16-byte aligned
    assert lib.sssgs_colors_to_image_bwd(h, 0, A, A, None) == INVALID


def _prototypes():
    """name -> (parameter count, return type) of every prototype in the header."""
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for m in re.finditer(r"\b([A-Za-z_][A-Za-z0-9_]*(?:\s*\*)?)\s+(sssgs_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", src):
        ret, name, params = m.group(1).strip(), m.group(2), m.group(3).strip()
        n = 0 if params in ("", "void") else params.count(",") + 1
        out[name] = (n, ret)
    return out


def test_binding_signatures_match_the_header_prototypes():
    """Every ctypes signature of the binding has the header's parameter count
    and a return type of the header's kind (int codes, sizes, strings)."""
    protos = _prototypes()
    assert set(protos) == set(_declared())
    kinds = {"int": ctypes.c_int, "size_t": ctypes.c_size_t, "int64_t": ctypes.c_int64,
             "uint64_t": ctypes.c_uint64, "void": None}
    for name, (args, res) in B._SIGS.items():
        n, ret = protos[name]
        assert len(args) == n, (name, len(args), n)
        if ret.replace(" ", "") == "char*":          # const char* (the qualifier is not captured)
            assert res is ctypes.c_char_p, name
        else:
            assert res is kinds[ret], (name, ret, res)
