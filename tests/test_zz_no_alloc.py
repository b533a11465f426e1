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


def _compare(seed, n_pairs, N, tx, ty):
    cfg, table, rec, rect, n_inst = _inputs(seed, n_pairs, N, tx, ty)
    cap = n_inst + 17
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


def test_static_scratch_rejects_oversize_problems():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = B.load_library()
    cfg, table, rec, rect, n_inst = _inputs(103, 1, 1000, 8, 8)
    v, r, c, s = _outputs(table, 1024)
    rc = lib.sssgs_bin_sort_static(ctypes.byref(cfg), table.h, table.d.data_ptr(), 1, rec.data_ptr(),
                                   rect.data_ptr(), B.STATIC_MAX_INSTANCES + 1, v.data_ptr(), r.data_ptr(),
                                   c.data_ptr(), s.data_ptr(), None)
    assert rc == B.ERR_TOO_LARGE
    assert "static scratch" in B.strerror(rc)
