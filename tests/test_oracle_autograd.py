"""The oracle's hand-derived backward against an independent dense FP64
restatement of the render differentiated by torch autograd (tiny scenes,
every pixel, every parameter entry).

The restatement follows the paper's equations directly and shares nothing
with the oracle but the conventions: EWA projection (Eq. 1, Eq. 2), alpha and
front-to-back compositing with the stop rule (Eq. 3), deferred GGX / Lambert
shading and the SSS blend at the back-projected point (Eq. 4, Eq. 7). Every
Gaussian is tested at every pixel (no tiles, no rectangles). The discrete
decisions (which Gaussians count at a pixel, where compositing stops, the
alpha clamp) are constants of the differentiation, as in the oracle; pixels
whose decisions lie near a threshold get no upstream gradient.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
import scenegen as sg
from test_oracle_grad import _tiny

KEYS = ["mu", "log_s", "quat", "logit_o", "normal", "base", "rough", "metal", "sss"]


def _rotation(q):
    q = q / q.norm(dim=1, keepdim=True)
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    return torch.stack([
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        torch.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        torch.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], -2)


def _unit(v):
    return v / v.norm(dim=-1, keepdim=True)


def _shade(n_raw, b, rough, metal, sss, Ls, Lin, x, cam_centre, light):
    """Eq. 4 (GGX D, Schlick F, separable Smith V, Lambert) and the Eq. 7
    blend at points x: sss L_SSS + (1 - sss) (f_s + f_d) L_in max(n . w_i, 0)."""
    wo, wi = _unit(cam_centre[None, :] - x), _unit(light[None, :] - x)
    n = n_raw / torch.clamp(n_raw.norm(dim=1, keepdim=True), min=1e-12)
    h = _unit(wo + wi)
    dot = lambda u, v: (u * v).sum(1)
    no, ni = torch.clamp(dot(n, wo), min=0), torch.clamp(dot(n, wi), min=0)
    nh, vh = torch.clamp(dot(n, h), min=0), torch.clamp(dot(wo, h), min=0)
    a2 = rough ** 4
    D = a2 / (math.pi * (nh * nh * (a2 - 1) + 1) ** 2)
    V = 1 / ((no + torch.sqrt(a2 + (1 - a2) * no * no)) * (ni + torch.sqrt(a2 + (1 - a2) * ni * ni)))
    mb = metal[:, None]
    F0 = 0.04 * (1 - mb) + b * mb
    Fr = F0 + (1 - F0) * ((1 - vh) ** 5)[:, None]
    fs = D[:, None] * Fr * V[:, None]
    fd = (1 - mb) * b / math.pi
    s = sss[:, None]
    return s * Ls + (1 - s) * (fs + fd) * (Lin * ni)[:, None]


def dense_render(P, mlp_out, pair, cfg, per_gaussian=False):
    """P: dict of FP64 leaf tensors (scene parameters); mlp_out: N x 4 leaf.
    Returns the image (H*W x 3, row-major) and the number of contributions.
    per_gaussian: each Gaussian shaded at its own mean and the colours
    composited (the paper's "w/o Deferred" ablation) instead of Eq. 4 / 7 on
    the composited G-buffer."""
    dil, det_eps, z_near = cfg.dilation, cfg.det_eps, cfg.z_near
    a_min, a_max, T_min, A_eps = cfg.alpha_min, cfg.alpha_max, cfg.T_min, cfg.A_eps
    Rc = torch.tensor(np.asarray(pair.R, np.float64))
    tc = torch.tensor(np.asarray(pair.t, np.float64))
    fx, fy, cx, cy = pair.fx, pair.fy, pair.cx, pair.cy
    cam_centre = -(Rc.T @ tc)
    light = torch.tensor(np.asarray(pair.light, np.float64))
    # Eq. 1 / Eq. 2: world covariance, view transform, affine projection
    Rg = _rotation(P["quat"])
    S2 = torch.exp(2 * P["log_s"])
    Sig = Rg @ torch.diag_embed(S2) @ Rg.transpose(1, 2)
    t = P["mu"] @ Rc.T + tc
    tx, ty, tz = t[:, 0], t[:, 1], t[:, 2]
    zero = torch.zeros_like(tz)
    J = torch.stack([torch.stack([fx / tz, zero, -fx * tx / tz ** 2], -1),
                     torch.stack([zero, fy / tz, -fy * ty / tz ** 2], -1)], -2)
    M = J @ Rc
    S2d = M @ Sig @ M.transpose(1, 2) + dil * torch.eye(2, dtype=torch.float64)
    conic = torch.linalg.inv(S2d)
    m2 = torch.stack([fx * tx / tz + cx, fy * ty / tz + cy], -1)
    o = torch.sigmoid(P["logit_o"])
    det = torch.linalg.det(S2d)
    alive = (tz >= z_near) & (det > det_eps) & (o > a_min)
    # every pixel centre against every Gaussian
    jj, ii = torch.meshgrid(torch.arange(pair.H, dtype=torch.float64), torch.arange(pair.W, dtype=torch.float64),
                            indexing="ij")
    px = torch.stack([ii.reshape(-1) + 0.5, jj.reshape(-1) + 0.5], -1)           # P x 2
    d = m2[None, :, :] - px[:, None, :]                                          # P x N x 2
    p = 0.5 * torch.einsum("pni,nij,pnj->pn", d, conic, d)
    a_raw = o[None, :] * torch.exp(-p)
    alpha = torch.minimum(a_raw, torch.full_like(a_raw, a_max))
    use = (p >= 0) & (alpha >= a_min) & alive[None, :]
    # Eq. 3: front to back in view depth (no near-ties: asserted by the caller)
    order = torch.argsort(tz.detach(), stable=True)
    feat = torch.cat([tz[:, None], P["normal"], P["base"], P["rough"][:, None], P["metal"][:, None],
                      P["sss"][:, None], mlp_out[:, :3], mlp_out[:, 3:4], P["vis"][:, None]], 1)
    if per_gaussian:
        col = _shade(P["normal"], P["base"], P["rough"], P["metal"], P["sss"], mlp_out[:, :3], mlp_out[:, 3],
                     P["mu"], cam_centre, light)
        feat = torch.cat([col, torch.zeros(col.shape[0], 12, dtype=torch.float64)], 1)
    npx = px.shape[0]
    T = torch.ones(npx, dtype=torch.float64)
    F = torch.zeros(npx, 15, dtype=torch.float64)
    running = torch.ones(npx, dtype=torch.bool)
    ncontrib = torch.zeros(npx, dtype=torch.int64)
    for g in order.tolist():
        a = alpha[:, g]
        Tn = T * (1 - a)
        takes = running & use[:, g]
        stop = takes & (Tn.detach() < T_min)                  # stop before this Gaussian
        running = running & ~stop
        takes = takes & ~stop
        w = torch.where(takes, T * a, torch.zeros_like(T))
        F = F + w[:, None] * feat[g][None, :]
        T = torch.where(takes, Tn, T)
        ncontrib = ncontrib + takes.long()
    has = ncontrib > 0
    rows = has.nonzero()[:, 0]
    if per_gaussian:                # colours composited as they are, black background
        return torch.zeros(npx, 3, dtype=torch.float64).index_put((rows,), F[has][:, 0:3]), ncontrib
    # Eq. 4, Eq. 7 at the back-projected point of the normalised G-buffer, on
    # the pixels something was composited into (the rest stay black)
    A = 1 - T[has]
    Ad = torch.maximum(A, torch.full_like(A, A_eps))
    g = F[has] / Ad[:, None]
    q = px[has]
    ray = torch.stack([(q[:, 0] - cx) / fx, (q[:, 1] - cy) / fy, torch.ones(q.shape[0], dtype=torch.float64)], -1)
    x = (g[:, 0:1] * ray - tc[None, :]) @ Rc                                   # R^T (d ray - t)
    L = _shade(g[:, 1:4], g[:, 4:7], g[:, 7], g[:, 8], g[:, 9], g[:, 10:13], g[:, 13], x, cam_centre, light)
    img = torch.zeros(npx, 3, dtype=torch.float64).index_put((rows,), A[:, None] * L)
    return img, ncontrib


@pytest.mark.parametrize("seed,opaque", [(0, False), (1, False), (2, False), (3, True), (4, True)])
def test_oracle_gradients_equal_dense_autograd(seed, opaque):
    """opaque: opacities pushed up so that alphas clamp at alpha_max and
    compositing stops on T < T_min at many pixels."""
    _check(seed, opaque, per_gaussian=False)


@pytest.mark.parametrize("seed,opaque", [(5, False), (3, True)])
def test_per_gaussian_shading_gradients_equal_dense_autograd(seed, opaque):
    """The "w/o Deferred" ablation path: colours from each Gaussian's own
    attributes at its mean, composited; the oracle's gradients (autograd of
    its colour function chained with the hand-derived compositing backward)
    against the dense restatement."""
    _check(seed, opaque, per_gaussian=True)


def _check(seed, opaque, per_gaussian):
    sc, pair, spec = _tiny(seed, N=30, log_s_mean=-1.1 if opaque else -1.8, res=40 if opaque else 32)
    if opaque:
        sc.logit_o = sc.logit_o + 8.0
    cfg = O.DEFAULT_CFG
    rng = np.random.default_rng(seed + 40)
    mlp_out = np.concatenate([rng.uniform(0, 1, (sc.N, 3)), rng.uniform(0, 2, (sc.N, 1))], 1)
    ref0 = O.render_pair(sc, pair, spec, mode=0, mlp_out=mlp_out, per_gaussian_shading=per_gaussian)
    # no two depths within float32 reach of each other: both sides order alike
    z = np.sort(ref0["proj"][:, 6])
    assert np.all(np.diff(z) > 1e-5 * np.abs(z[1:]))
    flag = (ref0["margin"][:, 0] < 2e-4) | (ref0["margin"][:, 1] < 5e-4)
    dimg = sg.random_dimg(seed + 90, pair.W * pair.H)
    dimg[flag] = 0.0
    ref = O.render_pair(sc, pair, spec, mode=0, mlp_out=mlp_out, dimg=dimg, per_gaussian_shading=per_gaussian)
    P = {k: torch.tensor(np.asarray(getattr(sc, k), np.float64), requires_grad=True) for k in KEYS + ["vis"]}
    mo = torch.tensor(mlp_out, requires_grad=True)
    img, nc = dense_render(P, mo, pair, cfg, per_gaussian=per_gaussian)
    assert np.array_equal(nc.numpy(), ref0["ncontrib"])
    np.testing.assert_allclose(img.detach().numpy(), ref0["img"], rtol=1e-9, atol=1e-12)
    (img * torch.tensor(dimg)).sum().backward()
    assert (ref0["ncontrib"] > 0).mean() > 0.3 and (~flag).mean() > 0.9
    if opaque:      # the clamp and the stop rule are exercised
        assert (ref0["margin"][:, 2] > 0).sum() >= 20
        assert (ref0["gbuf"][:, 15] < 1e-3).sum() >= 300
    for k in KEYS:
        got, want = ref["grads"][k], P[k].grad.numpy()
        err = np.linalg.norm(got - want) / max(np.linalg.norm(want), 1e-300)
        assert err < 1e-12, (k, err)
    assert not ref["grads"]["vis"].any()                                 # v does not enter the shading
    assert P["vis"].grad is None or not P["vis"].grad.any()
    err = np.linalg.norm(ref["dmlp_out"] - mo.grad.numpy()) / np.linalg.norm(mo.grad.numpy())
    assert err < 1e-12, err
