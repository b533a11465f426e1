"""Degenerate cases of the later rows on the GPU, through the C ABI:
* many lights per view and per-Gaussian shading with every Gaussian culled:
  black images, untouched transmittance, all gradients exactly zero;
* the visibility tracer over a scene of Gaussians below the alpha floor:
  nothing occludes, every v is exactly 1; a lone Gaussian sees its light;
* the image loss of an image against itself: SSIM = 1 and L1 = 0, so the loss
  and its gradient vanish up to FP32 cancellation.
"""
from dataclasses import replace

import numpy as np
import pytest
import torch

import scenegen as sg
from paper_2408_12282_gb300 import binding as B
from paper_2408_12282_gb300 import pipeline as PL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib(gpu_lib):
    return gpu_lib


def _far_away(wl):
    """Every Gaussian 50 units above the scene: off-screen or behind every camera."""
    wl.scenes = [replace(s, mu=s.mu + np.array([0.0, 0.0, 50.0])) for s in wl.scenes]
    return wl


def test_multilight_all_culled_is_black_with_zero_gradients():
    wl = _far_away(sg.make_workload("c6", N=64, res=32, n_views=2, n_lights=4))
    r = PL.multilight_renderer_for_workload(wl, precision=B.FP32)
    assert r.fit_capacity() == 0
    r.forward()
    P = r.img.shape[0]
    r.backward(dimg=torch.from_numpy(np.ascontiguousarray(sg.random_dimg(3, P), np.float32)).cuda())
    torch.cuda.synchronize()
    r.check_status()
    assert not r.img.any()
    assert torch.all(r.gbuf[:, 11] == 1.0)                 # final transmittance of an empty pixel
    assert all(not g.any() for g in r.grads.values())
    assert all(not g.any() for g in r.dW + r.db)


def test_per_gaussian_shading_all_culled_is_black_with_zero_gradients():
    wl = _far_away(sg.make_workload("c1", N=64, res=32))
    r = PL.renderer_for_workload(wl, precision=B.FP32, shading="gaussian")
    assert r.fit_capacity() == 0
    r.forward()
    r.backward(dimg=torch.from_numpy(np.ascontiguousarray(sg.random_dimg(4, 32 * 32), np.float32)).cuda())
    torch.cuda.synchronize()
    r.check_status()
    assert not r.img.any()
    assert all(not g.any() for g in r.grads.values())


@pytest.mark.parametrize("N", [1, 37, 3000])
def test_trace_through_transparent_gaussians_sees_the_light(N):
    """Opacity sigmoid(-10) = 4.5e-5 is below the alpha floor 1/255, so no
    Gaussian occludes: v = 1 for every (pair, Gaussian); N = 1 has no
    occluder at all (the BVH is a single leaf)."""
    wl = sg.make_workload("c4", N=N, res=32, n_pairs=3)
    wl.scenes[0] = replace(wl.scenes[0], logit_o=np.full(N, -10.0))
    r = PL.renderer_for_workload(wl, precision=B.FP32, vis_sh=sg.vis_sh_coeffs(1, N))
    v = r.trace_visibility()
    torch.cuda.synchronize()
    r.check_status()
    assert v.shape[0] == 3 * N
    assert torch.all(v == 1.0)


@pytest.mark.parametrize("tile", [8, 16])
def test_image_loss_of_identical_images_vanishes(tile):
    sizes = [(45, 37), (1, 1), (16, 16)]
    cfg = PL.default_cfg(tile)
    pairs = [sg.Pair(R=np.eye(3), t=np.zeros(3), fx=1.0, fy=1.0, cx=0, cy=0, W=w, H=h, light=np.zeros(3))
             for w, h in sizes]
    table = PL.PairTable(pairs, cfg, [0], [1])
    P = table.n_pixels
    img = torch.from_numpy(np.random.default_rng(tile).uniform(0, 1, (P, 3)).astype(np.float32)).cuda()
    dimg = torch.full((P, 3), float("nan"), device="cuda")
    loss = torch.zeros(len(sizes), device="cuda")                 # the loss accumulates (caller-zeroed)
    ws = torch.empty(B.image_loss_workspace_bytes(P), dtype=torch.uint8, device="cuda")
    B.image_loss(cfg, table.h, table.d, img, img.clone(), 0.2, dimg, loss, ws)
    torch.cuda.synchronize()
    off = 0
    for p, (w, h) in enumerate(sizes):
        n = 3 * w * h
        g = dimg[off:off + w * h].abs().max().item()
        # a gradient entry of a differing image is O(1 / n); here only rounding remains
        assert g <= 1e-5 / n, (p, g)
        assert abs(loss[p].item()) <= 1e-5, (p, loss[p].item())
        off += w * h
