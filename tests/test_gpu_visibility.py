"""Ray-traced visibility (BVH) and the SH visibility term on the GPU, through
the C ABI, against the oracle (oracle/visibility.py):
* traced visibility of every (pair, Gaussian) vs brute force over all
  Gaussians (items whose decisions lie within float32 reach of a threshold
  are excluded), one and two scenes (occluders only from the pair's scene);
* SH visibility forward and backward; the ray-traced visibility loss;
* a whole training step with the SH term (v evaluated per pair at the light
  direction) and the visibility loss against the oracle's render_pair fed the
  same per-pair v, with the chain rule through the SH term.
"""
from dataclasses import replace

import numpy as np
import pytest
import torch

import oracle as O
import oracle.visibility as V
import scenegen as sg
from gpu_common import assert_grads_close, assert_image_close, flagged
from paper_2408_12282_gb300 import binding as B
from paper_2408_12282_gb300 import pipeline as PL

pytestmark = pytest.mark.gpu

SCENE_KEYS = PL.SCENE_KEYS


@pytest.fixture(scope="module", autouse=True)
def _lib(gpu_lib):
    return gpu_lib


def _rel(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def _traced(wl):
    r = PL.renderer_for_workload(wl, precision=B.FP32, vis_sh=sg.vis_sh_coeffs(1, sum(s.N for s in wl.scenes)))
    v = r.trace_visibility()
    torch.cuda.synchronize()
    return r, v.double().cpu().numpy()


# Decision margins: float32 puts q* and t* within ~1e-6 (relative) of their
# FP64 values, so an item is excluded when one of its decisions lies within
# 2e-5 (relative) of its threshold.
MARGIN = 2e-5


@pytest.mark.parametrize("N,n_pairs,log_s_shift", [(3000, 3, -1.5), (3000, 2, -2.0), (3000, 1, 0.0),
                                                   (1, 1, 0.0), (40, 2, 0.0)])
def test_trace_matches_brute_force(N, n_pairs, log_s_shift):
    """Shifted scales give a shell with partly visible Gaussians (mean v 0.14
    and 0.39); the unshifted 3,000-Gaussian shell occludes nearly every ray
    (the tracer stops below 1e-5)."""
    wl = sg.make_workload("c4", N=N, res=32, n_pairs=n_pairs)
    wl.scenes[0] = replace(wl.scenes[0], log_s=wl.scenes[0].log_s + log_s_shift)
    r, got = _traced(wl)
    off = 0
    errs, excluded = [], 0
    for pair in wl.pairs:
        sc = wl.scenes[pair.scene]
        ref, margin = V.trace_visibility(sc, pair.light)
        ok = (margin > MARGIN) | (ref < 1e-4)        # a flip cannot move a v below 1e-4 by more than 1e-4
        excluded += int((~ok).sum())
        errs.append(np.abs(got[off:off + sc.N] - ref)[ok])
        off += sc.N
    err = np.concatenate(errs)
    print(f"\nN={N}: traced visibility max |gpu - oracle| {err.max() if err.size else 0:.2e}, "
          f"{excluded} items excluded, mean v {got.mean():.3f}")
    assert excluded <= max(1, 0.02 * got.size)
    assert err.size == 0 or err.max() <= 1e-4


def test_trace_two_scenes_do_not_occlude_each_other():
    wl = sg.make_workload("c5", N=2000, res=32, n_pairs=1)       # 8 scenes, one pair each
    wl.scenes, wl.pairs = wl.scenes[:2], wl.pairs[:2]
    r, got = _traced(wl)
    off = 0
    for pair in wl.pairs:
        sc = wl.scenes[pair.scene]
        ref, margin = V.trace_visibility(sc, pair.light)
        ok = (margin > MARGIN) | (ref < 1e-4)
        assert np.abs(got[off:off + sc.N] - ref)[ok].max() <= 1e-4
        off += sc.N


def test_vis_sh_forward_backward_and_loss():
    wl = sg.make_workload("c4", N=5000, res=32, n_pairs=3)
    sh = sg.vis_sh_coeffs(2, wl.scenes[0].N)
    r = PL.renderer_for_workload(wl, precision=B.FP32, vis_sh=sh)
    t = r.table
    B.vis_sh_fwd(t.h, t.d, r._scene_s, r.vis_sh, r.vis_item)
    rng = np.random.default_rng(3)
    dv = rng.uniform(-1, 1, t.n_items).astype(np.float32)
    vt = rng.uniform(0, 1, t.n_items).astype(np.float32)
    r.dvis_item.copy_(torch.from_numpy(dv))
    vt_d = torch.from_numpy(vt).cuda()
    loss = torch.zeros(t.n, device="cuda")
    B.vis_loss(t.h, t.d, r.vis_item, vt_d, 0.01, r.dvis_item, loss)
    dsh = torch.zeros_like(r.vis_sh)
    dmu = torch.zeros_like(r.scene["mu"])
    B.vis_sh_bwd(t.h, t.d, r._scene_s, r.vis_sh, r.dvis_item, dsh, dmu)
    torch.cuda.synchronize()
    v = r.vis_item.double().cpu().numpy()
    sc = wl.scenes[0]
    rdc = np.zeros_like(sh)
    rdmu = np.zeros_like(sc.mu)
    off = 0
    for p, pair in enumerate(wl.pairs):
        rv, u = V.vis_sh(sh, sc.mu, pair.light)
        np.testing.assert_allclose(v[off:off + sc.N], rv, atol=2e-6)
        lp, g = V.vis_loss(rv, vt[off:off + sc.N])
        assert abs(float(loss[p]) - lp) <= 1e-5 * lp
        dc, dm = V.vis_sh_backward(dv[off:off + sc.N] + g, sh, sc.mu, pair.light)
        rdc += dc
        rdmu += dm
        off += sc.N
    print(f"\nSH visibility: dsh rel-L2 {_rel(dsh.cpu().numpy(), rdc):.1e}, dmu {_rel(dmu.cpu().numpy(), rdmu):.1e}")
    assert _rel(dsh.cpu().numpy(), rdc) < 1e-5
    assert _rel(dmu.cpu().numpy(), rdmu) < 1e-5


def test_whole_step_with_sh_visibility_and_loss():
    wl = sg.make_workload("c2", N=8000, res=64, net="paper")   # the paper's network takes v as an input
    pair, sc = wl.pairs[0], wl.scenes[0]
    sh = sg.vis_sh_coeffs(4, sc.N)
    # oracle: v of this pair from the SH term, the renderer fed that v
    v_pair, _ = V.vis_sh(sh, sc.mu, pair.light)
    sc_v = replace(sc, vis=sg.f32(v_pair))
    ref0 = O.render_pair(sc_v, pair, wl.mlp, O.Cfg(tile=wl.tile))
    fl = flagged(ref0["margin"])
    dimg = sg.random_dimg(91, ref0["img"].shape[0])
    dimg[fl] = 0.0
    # the loss target: the oracle's traced visibility, given to both sides
    vt_np, _ = V.trace_visibility(sc, pair.light)
    vt_np = sg.f32(vt_np)
    r = PL.renderer_for_workload(wl, precision=B.FP32, vis_sh=sh)
    r.fit_capacity()
    r.vis_traced = torch.from_numpy(np.ascontiguousarray(vt_np, np.float32)).cuda()
    r.forward()
    r.backward(dimg=torch.from_numpy(np.ascontiguousarray(dimg, np.float32)).cuda(), lambda_raytrace=0.01)
    torch.cuda.synchronize()
    r.check_status()
    Lvis, dv_loss = V.vis_loss(v_pair, vt_np)
    ref = O.render_pair(sc_v, pair, wl.mlp, O.Cfg(tile=wl.tile), dimg=dimg, dvis_extra=dv_loss)
    dc, dmu = V.vis_sh_backward(ref["grads"]["vis"], sh, sc.mu, pair.light)
    ref_g = dict(ref["grads"])
    ref_g["mu"] = ref_g["mu"] + dmu
    assert_image_close(r.img.double().cpu().numpy(), ref0["img"], fl)
    got = {k: v.double().cpu().numpy() for k, v in r.grads.items()}
    keys = [k for k in SCENE_KEYS if k != "vis"]
    rep = assert_grads_close(got, ref_g, keys)
    assert not got["vis"].any()                       # v lives in the SH term here
    e = _rel(r.dvis_sh.cpu().numpy(), dc)
    print(f"\nstep with SH visibility: dsh rel-L2 {e:.1e}; loss {float(r.loss_vis[0]):.6f} vs {Lvis:.6f};",
          {k: f"{v[0]:.1e}" for k, v in rep.items()})
    assert e < 1e-3
    assert abs(float(r.loss_vis[0]) - Lvis) <= 1e-4 * max(Lvis, 1e-6)
