"""Many lights per view (sssgs_render_ml_fwd/bwd) on the GPU, through the C ABI.

A light-stage batch (scenegen c6: views under several lights of the 112-light
stage) must give, for every (view, light) pair, the image and the gradients
of rendering that pair on its own:
* against the FP64 oracle, pair by pair (images; every scene gradient and the
  network gradients summed over the batch);
* against the single-light path on the same pairs (same arithmetic per
  channel: images equal to float rounding, gradients to summation order);
* the weighted (IBL) forward equals the weighted sum of the per-light images;
* the fused L1 upstream equals an explicit dimg of l1_scale * sign(img - target).
"""
import numpy as np
import pytest
import torch

import scenegen as sg
from gpu_common import assert_grads_close, assert_image_close, flagged, oracle_batch
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


def _run_ml(wl, precision, dimg=None, target=None, l1_scale=1.0):
    r = PL.multilight_renderer_for_workload(wl, precision=precision)
    r.fit_capacity()
    r.forward()
    d = torch.from_numpy(np.ascontiguousarray(dimg, np.float32)).cuda() if dimg is not None else None
    t = torch.from_numpy(np.ascontiguousarray(target, np.float32)).cuda() if target is not None else None
    if d is not None or t is not None:
        r.backward(dimg=d, target=t, l1_scale=l1_scale)
    torch.cuda.synchronize()
    r.check_status()
    return r


@pytest.mark.parametrize("L", [1, 2, 4, 8])
def test_multilight_matches_oracle(L):
    wl = sg.make_workload("c6", N=12000, res=48, n_views=2, n_lights=L)
    ids = list(range(len(wl.pairs)))
    ref0 = oracle_batch(wl, ids)
    fl = flagged(ref0["margin"])
    dimg = sg.random_dimg(60 + L, ref0["img"].shape[0])
    dimg[fl] = 0.0
    ref = oracle_batch(wl, ids, dimg=dimg)
    r = _run_ml(wl, B.FP32, dimg=dimg)
    assert_image_close(r.img.double().cpu().numpy(), ref0["img"], fl)
    got = {k: v.double().cpu().numpy() for k, v in r.grads.items()}
    rep = assert_grads_close(got, ref["grads"], SCENE_KEYS)
    errs = {f"W{l}": _rel(r.dW[l].cpu().numpy(), ref["dW"][l]) for l in range(len(ref["dW"]))}
    errs.update({f"b{l}": _rel(r.db[l].cpu().numpy(), ref["db"][l]) for l in range(len(ref["db"]))})
    print(f"\nL={L}: {int(fl.sum())} flagged px; scene grads",
          {k: f"{v[0]:.1e}" for k, v in rep.items()}, "net", {k: f"{v:.1e}" for k, v in errs.items()})
    assert all(v < 1e-3 for v in errs.values()), errs


def test_multilight_equals_single_light_path():
    wl = sg.make_workload("c6", N=20000, res=64, n_views=3, n_lights=4)
    P = sum(p.W * p.H for p in wl.pairs)
    dimg = sg.random_dimg(77, P)
    ml = _run_ml(wl, B.BF16, dimg=dimg)
    r = PL.renderer_for_workload(wl, precision=B.BF16)
    r.fit_capacity()
    r.forward()
    r.backward(dimg=torch.from_numpy(np.ascontiguousarray(dimg, np.float32)).cuda())
    torch.cuda.synchronize()
    r.check_status()
    # same network rows (the pair table is the same), same compositing order
    assert torch.equal(ml.mlp_out, r.mlp_out)
    d = (ml.img - r.img).abs().max().item()
    assert d <= 1e-6, d
    # gradients: FP32 sums in another order (per-warp reductions of one pixel
    # per lane here, two there; atomics), and the BF16 network backward rounds
    # its slightly different upstream values to bfloat16
    errs = {k: _rel(ml.grads[k].cpu().numpy(), r.grads[k].cpu().numpy()) for k in SCENE_KEYS}
    errs.update({f"net{i}": _rel(a.cpu().numpy(), b.cpu().numpy()) for i, (a, b) in enumerate(zip(ml.dW + ml.db,
                                                                                               r.dW + r.db))})
    print("\nmany-light vs single-light rel-L2:", {k: f"{v:.1e}" for k, v in errs.items()})
    assert all(v < 1e-4 for k, v in errs.items() if not k.startswith("net")), errs
    assert all(v < 1e-3 for k, v in errs.items() if k.startswith("net")), errs


def test_multilight_ibl_weighted_sum():
    wl = sg.make_workload("c6", N=20000, res=64, n_views=2, n_lights=8)
    ml = _run_ml(wl, B.FP32)
    V, L = 2, 8
    w = np.random.default_rng(5).uniform(0, 2, V * L).astype(np.float32)
    out = torch.zeros(ml.views.n_pixels, 3, device="cuda")
    ml.forward(env_w=torch.from_numpy(w).cuda(), out=out)
    torch.cuda.synchronize()
    per = ml.img.double().cpu().numpy().reshape(V, L, -1, 3)
    ref = np.einsum("vl,vlpc->vpc", w.reshape(V, L).astype(np.float64), per).reshape(-1, 3)
    got = out.double().cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max())


def test_multilight_fused_l1_equals_explicit_dimg():
    wl = sg.make_workload("c6", N=12000, res=48, n_views=2, n_lights=2)
    ml = _run_ml(wl, B.FP32)
    img = ml.img.cpu().numpy()
    target = np.clip(img + np.random.default_rng(3).normal(0, 0.05, img.shape), 0, 1).astype(np.float32)
    s = 1.0 / img.size
    a = _run_ml(wl, B.FP32, target=target, l1_scale=s)
    b = _run_ml(wl, B.FP32, dimg=(s * np.sign(img - target)).astype(np.float32))
    for k in SCENE_KEYS:
        assert _rel(a.grads[k].cpu().numpy(), b.grads[k].cpu().numpy()) < 1e-6, k


def test_multilight_with_sh_visibility_equals_single_light_path():
    """The SH visibility term per (view, light) pair with the ray-traced
    visibility loss: the many-light renderer against the single-light path on
    the same pairs (network outputs equal, gradients to summation order)."""
    wl = sg.make_workload("c6", N=12000, res=48, n_views=2, n_lights=4, net="paper")
    sh = sg.vis_sh_coeffs(3, wl.scenes[0].N)
    P = sum(p.W * p.H for p in wl.pairs)
    dimg = torch.from_numpy(sg.random_dimg(19, P).astype(np.float32)).cuda()
    ml = PL.multilight_renderer_for_workload(wl, precision=B.FP32, vis_sh=sh)
    ml.fit_capacity()
    vt = ml.trace_visibility().clone()
    ml.forward()
    ml.backward(dimg=dimg)
    r = PL.renderer_for_workload(wl, precision=B.FP32, vis_sh=sh)
    r.fit_capacity()
    r.vis_traced = vt
    r.forward()
    r.backward(dimg=dimg)
    torch.cuda.synchronize()
    ml.check_status()
    r.check_status()
    assert torch.equal(ml.vis_item, r.vis_item)
    assert torch.allclose(ml.mlp_out, r.mlp_out, rtol=0, atol=0)
    assert (ml.img - r.img).abs().max().item() <= 1e-6
    assert torch.allclose(ml.loss_vis, r.loss_vis, rtol=1e-6)
    errs = {k: _rel(ml.grads[k].cpu().numpy(), r.grads[k].cpu().numpy()) for k in SCENE_KEYS if k != "vis"}
    errs["vis_sh"] = _rel(ml.dvis_sh.cpu().numpy(), r.dvis_sh.cpu().numpy())
    print("\nmany-light with SH visibility vs single-light rel-L2:", {k: f"{v:.1e}" for k, v in errs.items()})
    assert all(v < 1e-4 for v in errs.values()), errs
