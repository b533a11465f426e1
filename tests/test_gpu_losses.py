"""Training losses of App. E on the GPU (through the C ABI) against the oracle.

* image loss (1 - 0.2) L1 + 0.2 (1 - SSIM): per-pair loss values and dL/dimg
  for the same input images on both sides, at several image sizes (ragged
  tiles) and tile edges;
* incident-light constraint: loss values and the gradients added to the
  records' L_in and v fields;
* a rendered image (flat black background, smooth regions: the FP32
  moments' cancellation case) through the image loss on both sides;
* a whole step with the constraint: render backward of the oracle's image-loss
  gradient, the incident term added to the records, network and projection
  backward, against the oracle's render_pair with the same extra terms;
* the pipeline's backward with loss="paper" equals the same calls made one
  by one (image loss -> render backward with that dimg -> incident loss).
"""
import numpy as np
import pytest
import torch

import oracle as O
import scenegen as sg
from gpu_common import assert_grads_close, flagged
from paper_2408_12282_gb300 import binding as B
from paper_2408_12282_gb300 import pipeline as PL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib(gpu_lib):
    return gpu_lib


def _pairs(sizes, tile):
    cfg = PL.default_cfg(tile)
    pairs = [sg.Pair(R=np.eye(3), t=np.zeros(3), fx=1.0, fy=1.0, cx=0, cy=0, W=w, H=h, light=np.zeros(3))
             for w, h in sizes]
    return cfg, PL.PairTable(pairs, cfg, [0], [1])


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_image_loss_matches_oracle(tile):
    sizes = [(45, 37), (64, 64), (23, 70), (1, 1), (3, 50)]
    cfg, table = _pairs(sizes, tile)
    rng = np.random.default_rng(tile)
    P = table.n_pixels
    img = rng.uniform(0, 1, (P, 3)).astype(np.float32)
    tgt = np.clip(img + rng.normal(0, 0.1, (P, 3)), 0, 1).astype(np.float32)
    d_img = torch.from_numpy(img).cuda()
    d_tgt = torch.from_numpy(tgt).cuda()
    dimg = torch.full((P, 3), float("nan"), device="cuda")
    loss = torch.zeros(len(sizes), device="cuda")
    ws = torch.empty(B.image_loss_workspace_bytes(P), dtype=torch.uint8, device="cuda")
    B.image_loss(cfg, table.h, table.d, d_img, d_tgt, 0.2, dimg, loss, ws)
    torch.cuda.synchronize()
    g = dimg.double().cpu().numpy()
    lg = loss.double().cpu().numpy()
    off = 0
    for p, (w, h) in enumerate(sizes):
        n = w * h
        x = img[off:off + n].astype(np.float64).reshape(h, w, 3)
        y = tgt[off:off + n].astype(np.float64).reshape(h, w, 3)
        ref_loss, ref_g = O.image_loss(x, y)
        assert abs(lg[p] - ref_loss) <= 1e-5 * ref_loss, (p, lg[p], ref_loss)
        got = g[off:off + n].reshape(h, w, 3)
        rel = np.linalg.norm(got - ref_g) / np.linalg.norm(ref_g)
        print(f"\ntile {tile} pair {p} ({w}x{h}): loss {lg[p]:.6f} vs {ref_loss:.6f}, dimg rel-L2 {rel:.2e}")
        assert rel < 1e-4
        assert np.abs(got - ref_g).max() <= 1e-4 * np.abs(ref_g).max()
        off += n


def _image_loss_gpu(cfg, table, img, tgt):
    P = table.n_pixels
    dimg = torch.full((P, 3), float("nan"), device="cuda")
    loss = torch.zeros(table.n, device="cuda")
    ws = torch.empty(B.image_loss_workspace_bytes(P), dtype=torch.uint8, device="cuda")
    B.image_loss(cfg, table.h, table.d, torch.from_numpy(np.ascontiguousarray(img, np.float32)).cuda(),
                 torch.from_numpy(np.ascontiguousarray(tgt, np.float32)).cuda(), 0.2, dimg, loss, ws)
    torch.cuda.synchronize()
    return loss.double().cpu().numpy(), dimg.double().cpu().numpy()


def test_image_loss_on_rendered_image():
    wl = sg.make_workload("c2", N=20000, res=96)
    pair = wl.pairs[0]
    ref = O.render_pair(wl.scenes[0], pair, wl.mlp, O.Cfg(tile=wl.tile))
    H, W = pair.H, pair.W
    img = ref["img"].astype(np.float32)
    tgt = np.clip(img + np.random.default_rng(5).normal(0, 0.02, img.shape), 0, 1).astype(np.float32)
    tgt[:W * 8] = img[:W * 8]                      # top rows: identical (sign 0, SSIM 1 where flat)
    cfg, table = _pairs([(W, H)], wl.tile)
    lg, g = _image_loss_gpu(cfg, table, img, tgt)
    ref_loss, ref_g = O.image_loss(img.astype(np.float64).reshape(H, W, 3), tgt.astype(np.float64).reshape(H, W, 3))
    rel = np.linalg.norm(g.reshape(H, W, 3) - ref_g) / np.linalg.norm(ref_g)
    print(f"\nrendered image: loss {lg[0]:.7f} vs {ref_loss:.7f}, dimg rel-L2 {rel:.2e}")
    assert abs(lg[0] - ref_loss) <= 1e-5 * ref_loss
    assert rel < 1e-4


def test_whole_step_with_incident_constraint_matches_oracle():
    wl = sg.make_workload("c2", N=20000, res=96, net="paper")
    pair, sc = wl.pairs[0], wl.scenes[0]
    H, W = pair.H, pair.W
    ref0 = O.render_pair(sc, pair, wl.mlp, O.Cfg(tile=wl.tile))
    fl = flagged(ref0["margin"])
    tgt = np.clip(ref0["img"] + np.random.default_rng(9).normal(0, 0.05, ref0["img"].shape), 0, 1)
    _, gimg = O.image_loss(ref0["img"].reshape(H, W, 3), tgt.reshape(H, W, 3))
    dimg = gimg.reshape(-1, 3).copy()
    dimg[fl] = 0.0
    _, dl, dv = O.incident_loss(ref0["Lin"], sc.vis)
    ref = O.render_pair(sc, pair, wl.mlp, O.Cfg(tile=wl.tile), dimg=dimg, dlin_extra=dl, dvis_extra=dv)
    r = PL.renderer_for_workload(wl, precision=B.FP32)
    r.fit_capacity()
    r.forward()
    t = r.table
    r.zero_grads()
    loss = torch.zeros(t.n, device="cuda")
    d_dimg = torch.from_numpy(dimg.astype(np.float32)).cuda()
    B.render_bwd(r.cfg, t.h, t.d, r.rec, r.vals, r.ranges, r.gbuf, r.last, r.img, d_dimg, None, None, 1.0, r.drec)
    B.incident_loss(t.h, t.d, r.rec, 0.02, r.drec, loss)
    B.mlp_bwd(r._mlp_s, t.h, t.d, r._scene_s, r.drec, r._mlp_g, r.dx_items, r.ws_mlp, r.status)
    B.project_bwd(r.cfg, t.h, t.d, r._scene_s, r.drec, r.dx_items, r._grad_s)
    torch.cuda.synchronize()
    r.check_status()
    ref_inc, _, _ = O.incident_loss(ref0["Lin"], sc.vis)
    assert abs(float(loss[0]) - ref_inc) <= 1e-5 * ref_inc
    got = {k: v.double().cpu().numpy() for k, v in r.grads.items()}
    assert_grads_close(got, ref["grads"], PL.SCENE_KEYS)
    for l in range(6):
        a, b = r.dW[l].double().cpu().numpy(), ref["dW"][l]
        assert np.linalg.norm(a - b) <= 1e-3 * np.linalg.norm(b), l


def test_incident_loss_matches_oracle():
    wl = sg.make_workload("c4", N=3000, res=32, n_pairs=3)
    r = PL.renderer_for_workload(wl, precision=B.FP32)
    r.forward()
    r.zero_grads()
    d0 = r.drec.clone()
    loss = torch.zeros(r.table.n, device="cuda")
    B.incident_loss(r.table.h, r.table.d, r.rec, 0.02, r.drec, loss)
    torch.cuda.synchronize()
    rec = r.rec.double().cpu().numpy()
    dd = (r.drec - d0).double().cpu().numpy()
    lg = loss.double().cpu().numpy()
    off = 0
    for p, pair in enumerate(wl.pairs):
        n = wl.scenes[pair.scene].N
        ref_loss, dl, dv = O.incident_loss(rec[off:off + n, 19], rec[off:off + n, 20])
        assert abs(lg[p] - ref_loss) <= 2e-5 * ref_loss
        np.testing.assert_allclose(dd[off:off + n, 19], dl, rtol=1e-6, atol=1e-12)
        np.testing.assert_allclose(dd[off:off + n, 20], dv, rtol=1e-6, atol=1e-12)
        assert not np.delete(dd[off:off + n], [19, 20], axis=1).any()
        off += n


def test_pipeline_paper_loss_equals_calls_one_by_one():
    wl = sg.make_workload("c2", N=20000, res=96)
    target = torch.from_numpy(np.random.default_rng(3).uniform(0, 1, (96 * 96, 3)).astype(np.float32)).cuda()
    r = PL.renderer_for_workload(wl, precision=B.FP32)
    r.fit_capacity()
    r.forward()
    r.backward(target=target, loss="paper")
    torch.cuda.synchronize()
    got = {k: v.clone() for k, v in r.grads.items()}
    got_dW = [w.clone() for w in r.dW]
    got_loss = r.loss.clone()
    # the same step, one call at a time
    t = r.table
    r.zero_grads()
    dimg = torch.empty_like(r.img)
    loss = torch.zeros(t.n, device="cuda")
    ws = torch.empty(B.image_loss_workspace_bytes(t.n_pixels), dtype=torch.uint8, device="cuda")
    B.image_loss(r.cfg, t.h, t.d, r.img, target, 0.2, dimg, loss, ws)
    B.render_bwd(r.cfg, t.h, t.d, r.rec, r.vals, r.ranges, r.gbuf, r.last, r.img, dimg, None, None, 1.0, r.drec)
    B.incident_loss(t.h, t.d, r.rec, 0.02, r.drec, loss)
    B.mlp_bwd(r._mlp_s, t.h, t.d, r._scene_s, r.drec, r._mlp_g, r.dx_items, r.ws_mlp, r.status)
    B.project_bwd(r.cfg, t.h, t.d, r._scene_s, r.drec, r.dx_items, r._grad_s)
    torch.cuda.synchronize()
    assert torch.allclose(got_loss, loss, rtol=1e-6)
    for k in got:
        num = float((got[k] - r.grads[k]).norm())
        assert num <= 1e-5 * float(r.grads[k].norm()) + 1e-30, k
    for a, b in zip(got_dW, r.dW):
        assert float((a - b).norm()) <= 1e-5 * float(b.norm()) + 1e-30
    # the incident term moved L_in / v gradients: the loss includes it
    assert float(loss.sum()) > 0.0
