"""The allocation-free bin/sort entry point, for callers that cannot call
cudaMalloc (a plug-in whose host owns all device memory, a real-time loop that
cannot take cudaMalloc's device synchronisation): it must give exactly what the
workspace-based sssgs_bin_sort gives, call after call, although its scratch
keeps the previous call's contents. This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

import scenegen as sg
from paper_2408_12282_gb300 import binding as B
from paper_2408_12282_gb300 import pipeline as PL

pytestmark = pytest.mark.gpu


def _inputs(seed, n_pairs, N, tx, ty):
    rect, depth = sg.synthetic_bin_inputs(seed, n_pairs, N, tx, ty)
    cfg = PL.default_cfg(16)
    pairs = [sg.Pair(R=np.eye(3), t=np.zeros(3), fx=1.0, fy=1.0, cx=0, cy=0, W=tx * 16, H=ty * 16,
                     light=np.zeros(3)) for _ in range(n_pairs)]
    table = PL.PairTable(pairs, cfg, [0], [N])
    n = n_pairs * N
    rec = torch.zeros(n, B.REC, device="cuda")
    rec[:, 6] = torch.from_numpy(depth.astype(np.float32)).cuda()
    rect_t = torch.from_numpy(rect.astype(np.int32)).cuda()
    n_inst = int(((rect[:, 1] - rect[:, 0] + 1) * (rect[:, 3] - rect[:, 2] + 1) * (rect[:, 0] <= rect[:, 1])).sum())
    return cfg, table, rec, rect_t, n_inst


def _outputs(table, capacity):
    return (torch.full((capacity,), -1, dtype=torch.int32, device="cuda"),
            torch.full((table.n_tiles, 2), -1, dtype=torch.int32, device="cuda"),
            torch.zeros(1, dtype=torch.int64, device="cuda"),
            torch.zeros(1, dtype=torch.int32, device="cuda"))


def _compare(seed, n_pairs, N, tx, ty, cap=None):
    cfg, table, rec, rect, n_inst = _inputs(seed, n_pairs, N, tx, ty)
    cap = n_inst + 17 if cap is None else cap
    assert cap <= B.STATIC_MAX_INSTANCES and table.n_items <= B.STATIC_MAX_ITEMS
    v0, r0, c0, s0 = _outputs(table, cap)
    ws = torch.empty(B.bin_workspace_bytes(table.n_items, cap, table.n_tiles), dtype=torch.uint8, device="cuda")
    B.bin_sort(cfg, table.h, table.d, rec, rect, cap, v0, r0, c0, s0, ws)
    v1, r1, c1, s1 = _outputs(table, cap)
    B.bin_sort_static(cfg, table.h, table.d, rec, rect, cap, v1, r1, c1, s1)
    torch.cuda.synchronize()
    assert int(c1.item()) == int(c0.item()) == n_inst
    assert int(s1.item()) == int(s0.item()) == 0
    assert torch.equal(v1[:n_inst], v0[:n_inst])
    assert torch.equal(r1, r0)


def test_static_scratch_bin_sort_matches_workspace_version_twice_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.load_library()
    _compare(101, 3, 9000, 30, 20)     # larger first ...
    _compare(102, 1, 2500, 12, 7)      # ... then smaller: stale scratch must not leak


def test_static_scratch_at_its_exact_limits():
    """65,536 items and a capacity of 524,288 instances: the largest problem
    the fixed scratch takes, still equal to the workspace version."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.load_library()
    _compare(104, 1, B.STATIC_MAX_ITEMS, 8, 8, cap=B.STATIC_MAX_INSTANCES)


def _call_raw(lib, cfg, table, rec, rect, cap, outs):
    v, r, c, s = outs
    return lib.sssgs_bin_sort_static(ctypes.byref(cfg), table.h, table.d.data_ptr(), table.n, rec.data_ptr(),
                                     rect.data_ptr(), cap, v.data_ptr(), r.data_ptr(), c.data_ptr(), s.data_ptr(),
                                     None)


def _untouched(outs):
    v, r, c, s = outs
    torch.cuda.synchronize()
    return (bool((v == -1).all()) and bool((r == -1).all()) and int(c.item()) == -7 and int(s.item()) == -9)


def _sentinel_outputs(table, capacity):
    v, r, c, s = _outputs(table, capacity)
    c.fill_(-7)
    s.fill_(-9)
    return v, r, c, s


def test_static_scratch_rejects_oversize_problems():
    """Too many instances or too many items: SSSGS_ERR_TOO_LARGE before any
    launch, every output left as it was."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = B.load_library()
    cfg, table, rec, rect, n_inst = _inputs(103, 1, 1000, 8, 8)
    outs = _sentinel_outputs(table, 1024)
    rc = _call_raw(lib, cfg, table, rec, rect, B.STATIC_MAX_INSTANCES + 1, outs)
    assert rc == B.ERR_TOO_LARGE
    assert "static scratch" in B.strerror(rc)
    assert _untouched(outs)
    cfg, table, rec, rect, n_inst = _inputs(105, 1, B.STATIC_MAX_ITEMS + 1, 8, 8)
    outs = _sentinel_outputs(table, 1024)
    assert _call_raw(lib, cfg, table, rec, rect, 1024, outs) == B.ERR_TOO_LARGE
    assert _untouched(outs)


def test_static_scratch_rejects_malformed_arguments():
    """A negative capacity: SSSGS_ERR_INVALID_ARG before any launch."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = B.load_library()
    cfg, table, rec, rect, n_inst = _inputs(106, 1, 500, 8, 8)
    outs = _sentinel_outputs(table, 1024)
    assert _call_raw(lib, cfg, table, rec, rect, -1, outs) == B.ERR_INVALID_ARG
    assert _untouched(outs)
