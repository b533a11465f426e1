"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Sizes: the 1,024-Gaussian 128x128 workload in full; the 100K blob reduced to
20K Gaussians at 256x256 (several tiles, ragged edges with 8x8/16x16 tiles
not dividing 250); multi-pair batches of the 300K configuration at reduced
size. Full-size checks live in test_gpu_fullsize.py.
"""
import numpy as np
import pytest
import torch

import oracle as O
import scenegen as sg
from gpu_common import (assert_grads_close, assert_image_close, assert_tile_lists_equal, flagged, oracle_batch,
                        run_gpu, IMG_TOL)
from paper_2408_12282_gb300 import binding as B
from paper_2408_12282_gb300 import pipeline as PL

pytestmark = pytest.mark.gpu

SCENE_KEYS = PL.SCENE_KEYS


@pytest.fixture(scope="module", autouse=True)
def _lib(gpu_lib):
    return gpu_lib


def _masked_dimg(wl, pair_ids, seed):
    ref = oracle_batch(wl, pair_ids)
    npx = ref["img"].shape[0]
    dimg = sg.random_dimg(seed, npx)
    dimg[flagged(ref["margin"])] = 0.0
    return ref, dimg


# ------------------------------------------------------------------ projection

def test_projection_records_match_oracle():
    wl = sg.make_workload("c2", N=20000, res=256)
    g = run_gpu(wl, backward=False)
    proj, rect, dkey = O.project(wl.scenes[0], wl.pairs[0], O.Cfg(tile=16))
    rec = g["rec"]
    valid = rect[:, 0] <= rect[:, 1]
    assert valid.mean() > 0.9
    # mean2d, conic, opacity, depth
    np.testing.assert_allclose(rec[valid, 0:2], proj[valid, 0:2], rtol=0, atol=2e-3)
    for c in (2, 3, 4):
        scale = np.abs(proj[valid, c]).max()
        assert np.abs(rec[valid, c] - proj[valid, c]).max() <= 1e-4 * scale
    np.testing.assert_allclose(rec[valid, 5], proj[valid, 5], rtol=1e-6)
    # float32 depth key is bit-exact (the ordering decision)
    assert np.array_equal(rec[valid, 6].astype(np.float32).view(np.uint32), dkey[valid])
    # the GPU tile rectangle contains the oracle's (it is padded for float32)
    grect = g["rect"]
    t = 16
    orc = np.stack([rect[:, 0] // t, rect[:, 1] // t, rect[:, 2] // t, rect[:, 3] // t], 1)
    assert np.all(grect[valid, 0] <= orc[valid, 0]) and np.all(grect[valid, 1] >= orc[valid, 1])
    assert np.all(grect[valid, 2] <= orc[valid, 2]) and np.all(grect[valid, 3] >= orc[valid, 3])
    # culling constants: 1/ca, 1/cc, padded support level ln(o / alpha_min)
    np.testing.assert_allclose(rec[valid, 21], 1.0 / proj[valid, 2], rtol=2e-4)
    np.testing.assert_allclose(rec[valid, 22], 1.0 / proj[valid, 4], rtol=2e-4)
    np.testing.assert_allclose(rec[valid, 23], 1.001 * proj[valid, 7] + 0.01, rtol=1e-5, atol=1e-5)
    # features copied verbatim
    np.testing.assert_array_equal(rec[:, 7:10], wl.scenes[0].normal)
    np.testing.assert_array_equal(rec[:, 13], wl.scenes[0].rough)


def test_fp32_mlp_matches_oracle():
    for name, kw in [("c1", {}), ("c2", dict(N=5000, res=64)), ("c4", dict(N=3000, res=64, n_pairs=3))]:
        wl = sg.make_workload(name, **kw)
        g = run_gpu(wl, backward=False)
        off = 0
        for pair in wl.pairs:
            sc = wl.scenes[pair.scene]
            X = O.mlp_inputs(wl.mlp.kind, sc.mu, sc.normal, sc.vis, pair.center, pair.light)
            _, _, Ls, Lin = O.mlp_forward(wl.mlp, X)
            got = g["mlp_out"][off:off + sc.N]
            np.testing.assert_allclose(got[:, :3], Ls, atol=2e-6)
            np.testing.assert_allclose(got[:, 3], Lin, atol=2e-5 * max(1.0, np.abs(Lin).max()))
            off += sc.N


# ------------------------------------------------------------------ bin / sort

def _bin_gpu(rect, depth, n_pairs, N, tiles_x, tiles_y, capacity):
    cfg = PL.default_cfg(16)
    pairs = []
    for p in range(n_pairs):
        pairs.append(sg.Pair(R=np.eye(3), t=np.zeros(3), fx=1.0, fy=1.0, cx=0, cy=0, W=tiles_x * 16,
                             H=tiles_y * 16, light=np.zeros(3)))
    table = PL.PairTable(pairs, cfg, [0], [N])
    n = n_pairs * N
    rec = torch.zeros(n, B.REC, device="cuda")
    rec[:, 6] = torch.from_numpy(depth.astype(np.float32)).cuda()
    rect_t = torch.from_numpy(rect.astype(np.int32)).cuda()
    vals = torch.zeros(max(capacity, 1), dtype=torch.int32, device="cuda")
    ranges = torch.zeros(table.n_tiles, 2, dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(B.bin_workspace_bytes(n, capacity, table.n_tiles), dtype=torch.uint8, device="cuda")
    B.bin_sort(cfg, table.h, table.d, rec, rect_t, capacity, vals, ranges, count, status, ws)
    torch.cuda.synchronize()
    return (vals.cpu().numpy().view(np.uint32), ranges.cpu().numpy().view(np.uint32), int(count.item()),
            int(status.item()), table)


@pytest.mark.parametrize("n_pairs,N,tx,ty", [(1, 3000, 13, 9), (5, 7001, 20, 17), (64, 2500, 50, 50)])
def test_bin_sort_bit_exact(n_pairs, N, tx, ty):
    rect, depth = sg.synthetic_bin_inputs(17 + n_pairs, n_pairs, N, tx, ty)
    n_inst = int(((rect[:, 1] - rect[:, 0] + 1) * (rect[:, 3] - rect[:, 2] + 1) * (rect[:, 0] <= rect[:, 1])).sum())
    vals, ranges, count, status, table = _bin_gpu(rect, depth, n_pairs, N, tx, ty, n_inst + 100)
    item_pair = np.repeat(np.arange(n_pairs), N)
    n, keys, ovals, oranges = O.bin_sort(item_pair, rect, depth.view(np.uint32), np.full(n_pairs, tx),
                                         np.arange(n_pairs) * tx * ty, n_pairs * tx * ty)
    assert count == n == n_inst and status == 0
    assert_tile_lists_equal(vals[:n], ranges, ovals, oranges, n)


@pytest.mark.parametrize("name,kw", [("c2", {}), ("c4", dict(n_pairs=4))])
def test_bin_sort_real_scene_bit_exact(name, kw):
    """Tile lists of real scenes: the GPU's own float32 tile rectangles and
    depth keys (the projection's output) fed to the oracle's plain stable sort
    give exactly the GPU's list for every tile. Binning is an integer function
    of those values, so the comparison is bit for bit: the 100K blob at
    512x512, and four pairs of the 300K 800x800 batch (12M instances)."""
    wl = sg.make_workload(name, **kw)
    r = PL.renderer_for_workload(wl, precision=B.FP32)
    n_gpu = r.fit_capacity()
    torch.cuda.synchronize()
    r.check_status()
    rect = r.rect.cpu().numpy()
    dkey = r.rec[:, 6].contiguous().cpu().numpy().view(np.uint32)
    h = r.table.h
    n_pairs = r.table.n
    item_pair = np.repeat(np.arange(n_pairs), [h[p].g_count for p in range(n_pairs)])
    tiles_x = np.array([h[p].tiles_x for p in range(n_pairs)])
    tile_off = np.array([h[p].tile_offset for p in range(n_pairs)])
    n, _, ovals, oranges = O.bin_sort(item_pair, rect, dkey, tiles_x, tile_off, r.table.n_tiles)
    live = rect[:, 0] <= rect[:, 1]
    assert live.mean() > 0.5 and n > 10 * n_pairs * 1000
    assert n == n_gpu
    assert_tile_lists_equal(r.vals[:n].cpu().numpy().view(np.uint32), r.ranges.cpu().numpy().view(np.uint32),
                            ovals, oranges, n)


def test_bin_sort_capacity_overflow_is_flagged_not_trapped():
    rect, depth = sg.synthetic_bin_inputs(3, 2, 2000, 10, 10)
    n_inst = int(((rect[:, 1] - rect[:, 0] + 1) * (rect[:, 3] - rect[:, 2] + 1) * (rect[:, 0] <= rect[:, 1])).sum())
    vals, ranges, count, status, _ = _bin_gpu(rect, depth, 2, 2000, 10, 10, n_inst // 2)
    assert count == n_inst
    assert status & B.STATUS_CAPACITY
    assert ranges.max() <= n_inst // 2


def test_bin_sort_empty_and_all_culled():
    rect = np.tile(np.array([[1, 0, 1, 0]], np.int32), (100, 1))
    depth = np.ones(100, np.float32)
    vals, ranges, count, status, _ = _bin_gpu(rect, depth, 1, 100, 4, 4, 64)
    assert count == 0 and status == 0 and not ranges.any()


# ------------------------------------------------------------------ forward image

@pytest.mark.parametrize("name,kw", [("c1", {}), ("c2", dict(N=20000, res=256))])
def test_forward_image_and_gbuffer_match_oracle(name, kw):
    wl = sg.make_workload(name, **kw)
    ref = oracle_batch(wl, [0])
    g = run_gpu(wl, backward=False)
    fl = flagged(ref["margin"])
    assert fl.mean() < 0.05
    assert_image_close(g["img"], ref["img"], fl)
    assert_image_close(g["gbuf"], ref["gbuf"], fl, what="gbuf")
    assert (ref["ncontrib"] > 0).mean() > 0.2


def test_tile_size_and_fusion_do_not_change_pixels():
    """Tiles and splat batches only prune and stage candidates; per-pixel
    arithmetic and order are the same, so the forward is bit-identical across
    8/16/32 tiles, batches of 32/64 splats, and fused/unfused kernels."""
    wl = sg.make_workload("c2", N=20000, res=200)
    base = run_gpu(wl, backward=False, tile=16)
    for tile, batch, fused in [(8, 32, True), (32, 32, True), (16, 32, False), (8, 64, True), (16, 64, True),
                               (32, 64, True), (32, 64, False)]:
        g = run_gpu(wl, backward=False, tile=tile, fused=fused, batch=batch)
        assert np.array_equal(g["img"], base["img"]), (tile, batch, fused)
        assert np.array_equal(g["gbuf"], base["gbuf"]), (tile, batch, fused)
        if tile == 16:                 # list positions: the same lists only for the same tile edge
            assert np.array_equal(g["last"], base["last"]), (tile, batch, fused)


@pytest.mark.parametrize("tile,batch", [(8, 32), (32, 32), (8, 64), (16, 64), (32, 64)])
def test_gradients_match_oracle_every_schedule(tile, batch):
    """The one-warp backward at every tile edge and splat batch (ragged
    200 x 200 image: 8/16/32 do not divide it evenly, or only at one edge)."""
    wl = sg.make_workload("c2", N=20000, res=200)
    ref0, dimg = _masked_dimg(wl, [0], seed=77)
    ref = oracle_batch(wl, [0], dimg=dimg)
    g = run_gpu(wl, dimg=dimg, tile=tile, batch=batch)
    assert_image_close(g["img"], ref0["img"], flagged(ref0["margin"]))
    assert_grads_close(g["grads"], ref["grads"], SCENE_KEYS)


def test_batched_pairs_equal_single_pair_runs():
    wl = sg.make_workload("c4", N=4000, res=96, n_pairs=6)
    batch = run_gpu(wl, backward=False)
    off = 0
    for p in range(6):
        one = run_gpu(wl, backward=False, pair_slice=slice(p, p + 1))
        npx = wl.pairs[p].W * wl.pairs[p].H
        assert np.array_equal(batch["img"][off:off + npx], one["img"])
        off += npx


def test_empty_scene_and_culled_gaussians_render_black():
    wl = sg.make_workload("c1", N=64, res=32)
    wl.scenes[0].mu = wl.scenes[0].mu + np.array([0.0, 0.0, 50.0])   # all far off-screen / behind
    g = run_gpu(wl, dimg=sg.random_dimg(1, 32 * 32))
    assert not g["img"].any()
    assert np.all(g["gbuf"][:, 15] == 1.0)
    assert all(not v.any() for v in g["grads"].values())


# ------------------------------------------------------------------ backward

@pytest.mark.parametrize("name,kw", [("c1", {}), ("c2", dict(N=20000, res=256))])
def test_gradients_match_oracle(name, kw):
    wl = sg.make_workload(name, **kw)
    ref0, dimg = _masked_dimg(wl, [0], seed=99)
    ref = oracle_batch(wl, [0], dimg=dimg)
    g = run_gpu(wl, dimg=dimg)
    assert_grads_close(g["grads"], ref["grads"], SCENE_KEYS)
    assert_grads_close({f"W{l}": w for l, w in enumerate(g["dW"])},
                       {f"W{l}": w for l, w in enumerate(ref["dW"])}, [f"W{l}" for l in range(len(g["dW"]))])
    assert_grads_close({f"b{l}": w for l, w in enumerate(g["db"])},
                       {f"b{l}": w for l, w in enumerate(ref["db"])}, [f"b{l}" for l in range(len(g["db"]))])


def test_gradients_batched_pe6_fp32():
    wl = sg.make_workload("c4", N=3000, res=96, n_pairs=4)
    ref0, dimg = _masked_dimg(wl, range(4), seed=5)
    ref = oracle_batch(wl, range(4), dimg=dimg)
    g = run_gpu(wl, dimg=dimg)
    assert_grads_close(g["grads"], ref["grads"], SCENE_KEYS)
    for l in range(len(g["dW"])):
        assert_grads_close({"W": g["dW"][l]}, {"W": ref["dW"][l]}, ["W"])


def test_unfused_backward_matches_fused():
    wl = sg.make_workload("c2", N=10000, res=128)
    dimg = sg.random_dimg(4, 128 * 128)
    a = run_gpu(wl, dimg=dimg, fused=True)
    b = run_gpu(wl, dimg=dimg, fused=False)
    assert_grads_close(a["grads"], b["grads"], SCENE_KEYS, tol=1e-5)


def test_fused_l1_loss_gradient():
    """dimg = scale * sign(img - target): the sign is taken from each side's own
    image; pixels where |img - target| is within float32 reach are masked."""
    wl = sg.make_workload("c1")
    pair = wl.pairs[0]
    tgt = O.render_pair(wl.target_scene, pair, wl.mlp)["img"]
    ref0 = oracle_batch(wl, [0])
    weight = np.ones(pair.W * pair.H)
    weight[flagged(ref0["margin"])] = 0.0
    weight[np.any(np.abs(ref0["img"] - tgt) < 1e-5, axis=1)] = 0.0
    scale = 1.0 / (3 * pair.W * pair.H)
    dimg = scale * weight[:, None] * np.sign(ref0["img"] - tgt)
    ref = oracle_batch(wl, [0], dimg=dimg)
    g = run_gpu(wl, target=tgt, weight=weight, l1_scale=scale)
    assert_grads_close(g["grads"], ref["grads"], SCENE_KEYS)


def test_autograd_function_matches_direct_backward():
    wl = sg.make_workload("c1")
    r = PL.renderer_for_workload(wl)
    r.fit_capacity()
    params = [r.scene[k] for k in SCENE_KEYS] + r.mlp.W + r.mlp.b
    for p in params:
        p.requires_grad_(True)
    img = PL.render(r)
    dimg = torch.from_numpy(sg.random_dimg(3, img.shape[0]).astype(np.float32)).cuda()
    (img * dimg).sum().backward()
    direct = {k: v.clone() for k, v in r.grads.items()}
    for k in SCENE_KEYS:
        assert torch.allclose(r.scene[k].grad, direct[k], rtol=0, atol=0)


def test_cuda_graph_replay_matches_eager_step():
    wl = sg.make_workload("c4", N=3000, res=64, n_pairs=3)
    r = PL.renderer_for_workload(wl, precision=B.FP32)
    r.fit_capacity()
    dimg = torch.from_numpy(sg.random_dimg(8, r.table.n_pixels).astype(np.float32)).cuda()
    r.forward()
    r.backward(dimg=dimg)
    torch.cuda.synchronize()
    eager_img = r.img.clone()
    eager = {k: v.clone() for k, v in r.grads.items()}
    g = r.capture(dimg=dimg)
    r.img.zero_()
    for v in r.grads.values():
        v.fill_(123.0)
    g.replay()
    torch.cuda.synchronize()
    r.check_status()
    assert torch.equal(r.img, eager_img)            # forward: deterministic, bit-identical
    for k in SCENE_KEYS:                             # backward: float atomics, order may differ
        num = float((r.grads[k] - eager[k]).norm())
        den = float(eager[k].norm())
        assert num <= 1e-5 * den, (k, num, den)


def test_work_counters():
    """Contribution counters of the fused kernels equal the oracle's count of
    composited (pixel, Gaussian) pairs (up to flagged decisions)."""
    wl = sg.make_workload("c2", N=20000, res=128)
    r = PL.renderer_for_workload(wl)
    r.fit_capacity()
    r.stats_fwd = torch.zeros(2, dtype=torch.int64, device="cuda")
    r.stats_bwd = torch.zeros(2, dtype=torch.int64, device="cuda")
    r.forward()
    r.backward(dimg=torch.ones(r.table.n_pixels, 3, device="cuda"))
    torch.cuda.synchronize()
    ref = oracle_batch(wl, [0])
    n_ref = int(ref["ncontrib"].sum())
    cf, ef = r.stats_fwd.tolist()
    cb, eb = r.stats_bwd.tolist()
    assert cf == cb
    assert abs(cf - n_ref) <= 0.001 * n_ref
    assert ef >= cf and eb >= cb


def test_uneven_batch_several_scenes_and_resolutions():
    """The uneven configuration shape: several scenes of different sizes, each
    with its own pairs, images of different sizes, one batch."""
    wl = sg.make_workload("c5", N=20000, res=(40, 64, 88), n_pairs=2)
    for p in wl.pairs:
        assert p.W in (40, 64, 88)
    pid = list(range(len(wl.pairs)))
    ref0, dimg = _masked_dimg(wl, pid, seed=31)
    ref = oracle_batch(wl, pid, dimg=dimg)
    g = run_gpu(wl, precision=B.FP32, dimg=dimg)
    fl = flagged(ref0["margin"])
    assert_image_close(g["img"], ref0["img"], fl)
    assert_grads_close(g["grads"], ref["grads"], SCENE_KEYS)
    assert len({(p.W, p.H) for p in wl.pairs}) > 1 and len(wl.scenes) == 8


def test_autotuner_picks_the_fastest_measured_candidate_per_scene():
    """sssgs_autotune through autotune_schedule on an uneven batch of 8 scenes:
    every (tile, batch) candidate of every scene is run and timed, and each
    scene's schedule is its fastest candidate."""
    wl = sg.make_workload("c5", N=20000, res=(40, 64, 88), n_pairs=2)
    cfgs, table = PL.autotune_schedule(wl, precision=B.FP32, reps=1)
    assert len(cfgs) == len(wl.scenes) == len(table)
    for sc, res in table.items():
        assert len(res) == 6 and {(x.tile, x.batch) for x in res} == {(t, b) for t in (8, 16, 32) for b in (32, 64)}
        assert all(x.status == 0 and x.ms > 0 and x.reps == 1 and x.instances > 0 for x in res)
        fastest = min(res, key=lambda x: x.ms)
        assert (cfgs[sc].tile, cfgs[sc].batch) == (fastest.tile, fastest.batch)
        # smaller tiles never give fewer instances
        inst = {x.tile: x.instances for x in res}
        assert inst[8] >= inst[16] >= inst[32]


def test_autotuner_reruns_candidates_that_exceed_the_first_capacity():
    """First trial buffers far too small for every candidate (no candidate
    fits: sssgs_autotune reports every instance count and returns
    SSSGS_ERR_WORKSPACE): the candidates are rerun with buffers sized from
    their counts, and the result is the same kind of complete table."""
    wl = sg.make_workload("c5", N=20000, res=(40, 64, 88), n_pairs=2)
    cfgs, table = PL.autotune_schedule(wl, precision=B.FP32, reps=1, instances_per_item=0.0)
    for sc, res in table.items():
        assert all(x.status == 0 and x.ms > 0 and x.instances > 0 for x in res)
        fastest = min(res, key=lambda x: x.ms)
        assert (cfgs[sc].tile, cfgs[sc].batch) == (fastest.tile, fastest.batch)


def test_per_scene_schedule_with_the_paper_losses():
    """The App. E training losses (image loss over the whole batch, then the
    per-run render backward) on a per-scene schedule: the same losses and
    gradients as with one schedule."""
    wl = sg.make_workload("c5", N=20000, res=(40, 64, 88), n_pairs=2)
    cfgs = []
    for sc in range(len(wl.scenes)):
        c = PL.default_cfg((8, 16, 32)[sc % 3])
        c.batch = (32, 64)[sc % 2]
        cfgs.append(c)
    ra = PL.renderer_for_workload(wl, precision=B.FP32, scene_cfgs=cfgs)
    rb = PL.renderer_for_workload(wl, precision=B.FP32)
    assert ra.groups is not None and rb.groups is None
    target = None
    for r in (ra, rb):
        r.fit_capacity()
        r.forward()
        if target is None:
            target = torch.rand_like(r.img)
        r.backward(target=target, loss="paper")
    torch.cuda.synchronize()
    ra.check_status()
    rb.check_status()
    assert torch.equal(ra.img, rb.img)
    assert torch.allclose(ra.loss, rb.loss, rtol=1e-5, atol=0)
    for k in SCENE_KEYS:
        num = float((ra.grads[k] - rb.grads[k]).norm())
        den = float(rb.grads[k].norm())
        assert num <= 1e-5 * max(den, 1e-30), (k, num, den)


def test_per_scene_schedule_matches_oracle_and_single_schedule():
    """A batch whose scenes run with different tile edges and batches (one run
    of pairs per scene, each on its own stream, one captured graph): the
    forward is bit-identical to the single-schedule batch and the gradients
    match the oracle."""
    wl = sg.make_workload("c5", N=20000, res=(40, 64, 88), n_pairs=2)
    pid = list(range(len(wl.pairs)))
    ref0, dimg = _masked_dimg(wl, pid, seed=41)
    ref = oracle_batch(wl, pid, dimg=dimg)
    cfgs = []
    for sc in range(len(wl.scenes)):
        c = PL.default_cfg((8, 16, 32)[sc % 3])
        c.batch = (32, 64)[(sc // 3) % 2]
        cfgs.append(c)
    g = run_gpu(wl, precision=B.FP32, dimg=dimg, scene_cfgs=cfgs)
    assert g["renderer"].groups is not None and len(g["renderer"].groups) == len(wl.scenes)
    single = run_gpu(wl, precision=B.FP32, backward=False)
    assert np.array_equal(g["img"], single["img"])
    assert_image_close(g["img"], ref0["img"], flagged(ref0["margin"]))
    assert_grads_close(g["grads"], ref["grads"], SCENE_KEYS)
    # the same step replayed from a captured graph
    r = g["renderer"]
    graph = r.capture(dimg=torch.from_numpy(dimg.astype(np.float32)).cuda())
    r.img.zero_()
    graph.replay()
    torch.cuda.synchronize()
    r.check_status()
    assert np.array_equal(r.img.double().cpu().numpy(), single["img"])
