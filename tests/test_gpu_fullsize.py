"""Full-size parity, in the launch configuration the benchmark times.

* The 300K-Gaussian 800x800 pair (tensor-core network, fused kernels): every
  pixel and every gradient tensor against the oracle with the BF16-emulating
  network (gates of test_gpu_tc: bf16 decision flips are the only expected
  differences).
* The 64-pair 300K batch replayed from a captured CUDA graph with the fused
  L1 loss, as in bench.py: sampled pixels of two pairs against the oracle, and
  those pairs bit-identical to single-pair renders.
* The same for the light-stage batch, the uneven batch of 50K-1M Gaussian
  scenes at 400-1600 px, and the ray-traced visibility of the 64-pair batch.
"""
import numpy as np
import pytest
import torch

import oracle as O
import scenegen as sg
from gpu_common import flagged, grad_errors, oracle_batch, run_gpu
from paper_2408_12282_gb300 import binding as B
from paper_2408_12282_gb300 import pipeline as PL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib(gpu_lib):
    return gpu_lib


def test_full_300k_800_pair_image_and_gradients():
    wl = sg.make_workload("c3")
    ref0 = oracle_batch(wl, [0], bf16=True)
    fl = flagged(ref0["margin"])
    dimg = sg.random_dimg(123, ref0["img"].shape[0])
    dimg[fl] = 0.0
    ref = oracle_batch(wl, [0], dimg=dimg, bf16=True)
    g = run_gpu(wl, precision=B.BF16, dimg=dimg)
    ok = ~fl
    e = np.abs(g["img"][ok] - ref0["img"][ok]).max(axis=1)
    print(f"\nfull 300K/800 pair: {fl.mean():.2%} flagged; image max {e.max():.2e} p99.9 {np.quantile(e, 0.999):.2e}")
    assert fl.mean() < 0.05
    assert np.quantile(e, 0.999) <= 1e-4 and e.max() <= 5e-3
    errs = {k: grad_errors(g["grads"][k], ref["grads"][k])[0] for k in PL.SCENE_KEYS}
    errs.update({f"W{l}": grad_errors(g["dW"][l], ref["dW"][l])[0] for l in range(len(g["dW"]))})
    print("gradient rel-L2:", {k: f"{v:.1e}" for k, v in errs.items()})
    assert all(v <= 2e-3 for v in errs.values()), errs


def test_full_64_pair_batch_graph_replay_sampled():
    wl = sg.make_workload("c4")
    r = PL.renderer_for_workload(wl, precision=B.BF16)
    r.fit_capacity()
    target = torch.zeros(r.table.n_pixels, 3, device="cuda")
    graph = r.capture(target=target, l1_scale=1.0 / (3.0 * r.table.n_pixels))
    graph.replay()
    graph.replay()
    torch.cuda.synchronize()
    r.check_status()
    img = r.img.double().cpu().numpy()
    rng = np.random.default_rng(5)
    off = 0
    offs = [0]
    for p in wl.pairs:
        offs.append(offs[-1] + p.W * p.H)
    for p in (7, 41):
        pair = wl.pairs[p]
        pix = O.all_pixels(pair.W, pair.H)
        sel = rng.choice(len(pix), 1500, replace=False)
        res = O.render_pair(wl.scenes[0], pair, wl.mlp, pixels=pix[sel].astype(np.int32), bf16=True)
        fl = flagged(res["margin"])
        got = img[offs[p] + sel]
        e = np.abs(got[~fl] - res["img"][~fl]).max(axis=1)
        print(f"\npair {p}: {fl.mean():.2%} flagged, max {e.max():.2e}, p99 {np.quantile(e, 0.99):.2e}")
        assert np.quantile(e, 0.99) <= 1e-4 and e.max() <= 5e-3
        one = PL.renderer_for_workload(wl, precision=B.BF16, pair_slice=slice(p, p + 1))
        one.fit_capacity()
        one.forward()
        torch.cuda.synchronize()
        assert torch.equal(one.img, r.img[offs[p]:offs[p + 1]])
        del one
        torch.cuda.empty_cache()


def test_full_light_stage_batch_graph_replay_sampled():
    """The 8 views x 8 lights light-stage batch (300K, 800x800) through the
    many-light kernels, replayed from a captured graph with the fused L1 loss
    as in bench.py: sampled pixels of two (view, light) pairs against the
    oracle rendering that pair on its own."""
    import oracle as O2
    wl = sg.make_workload("c6")
    r = PL.multilight_renderer_for_workload(wl, precision=B.BF16)
    r.fit_capacity()
    target = torch.zeros(r.pairs.n_pixels, 3, device="cuda")
    graph = r.capture(target=target, l1_scale=1.0 / (3.0 * r.pairs.n_pixels))
    graph.replay()
    graph.replay()
    torch.cuda.synchronize()
    r.check_status()
    img = r.img.double().cpu().numpy()
    assert np.isfinite(r.grads["mu"].cpu().numpy()).all()
    rng = np.random.default_rng(6)
    offs = [0]
    for p in wl.pairs:
        offs.append(offs[-1] + p.W * p.H)
    for p in (3, 58):                  # view 0 light 3, view 7 light 2
        pair = wl.pairs[p]
        pix = O2.all_pixels(pair.W, pair.H)
        sel = rng.choice(len(pix), 1500, replace=False)
        res = O2.render_pair(wl.scenes[0], pair, wl.mlp, pixels=pix[sel].astype(np.int32), bf16=True)
        fl = flagged(res["margin"])
        got = img[offs[p] + sel]
        e = np.abs(got[~fl] - res["img"][~fl]).max(axis=1)
        print(f"\nlight-stage pair {p}: {fl.mean():.2%} flagged, max {e.max():.2e}, p99 {np.quantile(e, 0.99):.2e}")
        assert np.quantile(e, 0.99) <= 1e-4 and e.max() <= 5e-3


def test_full_uneven_batch_graph_replay_sampled():
    """The uneven batch (8 scenes of 50K-1M Gaussians, 8 pairs each at
    400-1600 px) replayed from a captured graph with the fused L1 loss, as in
    bench.py: sampled pixels of the smallest scene's first image and of the
    1M-Gaussian scene's largest image against the oracle rendering that pair
    on its own."""
    wl = sg.make_workload("c5")
    r = PL.renderer_for_workload(wl, precision=B.BF16)
    r.fit_capacity()
    target = torch.zeros(r.table.n_pixels, 3, device="cuda")
    graph = r.capture(target=target, l1_scale=1.0 / (3.0 * r.table.n_pixels))
    graph.replay()
    graph.replay()
    torch.cuda.synchronize()
    r.check_status()
    img = r.img.double().cpu().numpy()
    assert all(torch.isfinite(g).all().item() for g in r.grads.values())
    offs = [0]
    for p in wl.pairs:
        offs.append(offs[-1] + p.W * p.H)
    small = next(p for p, q in enumerate(wl.pairs) if q.scene == 0)
    big = max((p for p, q in enumerate(wl.pairs) if q.scene == len(wl.scenes) - 1), key=lambda p: wl.pairs[p].W)
    rng = np.random.default_rng(8)
    for p in (small, big):
        pair = wl.pairs[p]
        pix = O.all_pixels(pair.W, pair.H)
        sel = rng.choice(len(pix), 1500, replace=False)
        res = O.render_pair(wl.scenes[pair.scene], pair, wl.mlp, pixels=pix[sel].astype(np.int32), bf16=True)
        fl = flagged(res["margin"])
        got = img[offs[p] + sel]
        e = np.abs(got[~fl] - res["img"][~fl]).max(axis=1)
        print(f"\nuneven batch pair {p} (scene {pair.scene}, {wl.scenes[pair.scene].N} Gaussians, {pair.W}x{pair.H}): "
              f"{fl.mean():.2%} flagged, max {e.max():.2e}, p99 {np.quantile(e, 0.99):.2e}")
        assert (res["ncontrib"] > 0).mean() > 0.05
        assert np.quantile(e, 0.99) <= 1e-4 and e.max() <= 5e-3


def test_full_batch_visibility_trace_sampled():
    """Ray-traced visibility of the 64-pair 300K batch: sampled items of two
    pairs against the oracle's brute force over all 300K Gaussians."""
    import oracle.visibility as V
    wl = sg.make_workload("c4")
    sc = wl.scenes[0]
    r = PL.renderer_for_workload(wl, precision=B.BF16, vis_sh=sg.vis_sh_coeffs(1, sc.N))
    v = r.trace_visibility()
    torch.cuda.synchronize()
    got = v.double().cpu().numpy()
    rng = np.random.default_rng(8)
    for p in (5, 50):
        items = rng.choice(sc.N, 60, replace=False)
        ref, margin = V.trace_visibility(sc, wl.pairs[p].light, items=items)
        ok = (margin > 2e-5) | (ref < 1e-4)
        e = np.abs(got[p * sc.N + items] - ref)[ok]
        print(f"\ntrace pair {p}: {int((~ok).sum())} excluded, max |gpu - oracle| {e.max():.2e}")
        assert (~ok).sum() <= 3 and e.max() <= 1e-4
