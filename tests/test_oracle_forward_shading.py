"""Pins of the oracle's per-Gaussian shading (the paper's "w/o Deferred"
ablation): the colour of a Gaussian equals the independent C deferred shading
of a pixel whose back-projected point is that Gaussian's mean; its autograd
gradient equals finite differences; a lone Gaussian at a pixel centre gives
o * c; brute force equals tiled; and the whole per-Gaussian-shaded render's
gradient equals central finite differences."""
import math
from dataclasses import replace

import numpy as np
import pytest

import oracle as O
import scenegen as sg
from test_oracle_grad import _tiny, PARAMS


def _feats(rng, n):
    normal = rng.normal(size=(n, 3))
    return dict(normal=normal, base=rng.uniform(0, 1, (n, 3)), rough=rng.uniform(0.1, 1, n),
                metal=rng.uniform(0, 1, n), sss=rng.uniform(0, 1, n), Ls=rng.uniform(0, 1, (n, 3)),
                Lin=rng.uniform(0, 2, n))


def test_colour_equals_deferred_shading_at_the_mean():
    """A pixel of A = 1 (T = 0) whose depth puts its back-projected point on a
    Gaussian's mean shades that Gaussian's features exactly as the per-Gaussian
    shading does (independent C implementation of Eq. 4 and Eq. 7)."""
    rng = np.random.default_rng(0)
    pair = sg.make_workload("c1", res=32).pairs[0]
    n = 40
    pix = np.stack([rng.integers(0, 32, n), rng.integers(0, 32, n)], 1).astype(np.int32)
    depth = rng.uniform(2.0, 4.0, n)
    ray = np.stack([(pix[:, 0] + 0.5 - pair.cx) / pair.fx, (pix[:, 1] + 0.5 - pair.cy) / pair.fy, np.ones(n)], 1)
    mu = (depth[:, None] * ray - pair.t[None, :]) @ pair.R          # x = R^T (d ray - t)
    f = _feats(rng, n)
    c = O.gaussian_colors(f["normal"], f["base"], f["rough"], f["metal"], f["sss"], f["Ls"], f["Lin"], mu,
                          pair.center, pair.light)
    gbuf = np.concatenate([depth[:, None], f["normal"], f["base"], f["rough"][:, None], f["metal"][:, None],
                           f["sss"][:, None], f["Ls"], f["Lin"][:, None], np.zeros((n, 1)), np.zeros((n, 1))], 1)
    img, _ = O.shade(gbuf, np.ones(n, np.int32), pix, pair)
    np.testing.assert_allclose(c, img, rtol=1e-10, atol=1e-12)


def test_colour_gradient_equals_finite_differences():
    rng = np.random.default_rng(1)
    n = 8
    f = _feats(rng, n)
    mu = rng.normal(0, 0.5, (n, 3))
    C, Lp = np.array([0.3, -2.5, 1.5]), np.array([2.0, 1.0, 3.0])
    g = rng.uniform(-1, 1, (n, 3))
    args = [f["normal"], f["base"], f["rough"], f["metal"], f["sss"], f["Ls"], f["Lin"], mu]
    _, grads = O.gaussian_colors(*args, C, Lp, grad_out=g)
    h = 1e-6
    for a_i, a in enumerate(args):
        flat = a.reshape(-1)
        for k in rng.choice(flat.size, min(6, flat.size), replace=False):
            x0 = flat[k]
            flat[k] = x0 + h
            fp = float((O.gaussian_colors(*args, C, Lp) * g).sum())
            flat[k] = x0 - h
            fm = float((O.gaussian_colors(*args, C, Lp) * g).sum())
            flat[k] = x0
            assert abs((fp - fm) / (2 * h) - grads[a_i].reshape(-1)[k]) <= 1e-6 * max(1.0, abs(grads[a_i].reshape(-1)[k]))


def test_lone_gaussian_composites_to_opacity_times_colour():
    sc, pair, spec = _tiny(2, N=1)
    sc = replace(sc, log_s=np.full((1, 3), -2.0), logit_o=np.array([0.4]))
    C = pair.center
    # put the Gaussian on the ray of pixel (10, 12) at depth 2.5
    ray = np.array([(10.5 - pair.cx) / pair.fx, (12.5 - pair.cy) / pair.fy, 1.0])
    sc = replace(sc, mu=((2.5 * ray - pair.t) @ pair.R)[None, :])
    cfg = replace(O.DEFAULT_CFG, dilation=0.0)
    r = O.render_pair(sc, pair, spec, cfg=cfg, pixels=np.array([[10, 12]], np.int32), per_gaussian_shading=True)
    o = 1 / (1 + math.exp(-0.4))
    c = O.gaussian_colors(sc.normal, sc.base, sc.rough, sc.metal, sc.sss, r["Ls"], r["Lin"], sc.mu, C, pair.light)
    np.testing.assert_allclose(r["img"][0], o * c[0], rtol=1e-10)


def test_brute_force_equals_tiled():
    sc, pair, spec = _tiny(3, N=60)
    a = O.render_pair(sc, pair, spec, mode=0, per_gaussian_shading=True)
    b = O.render_pair(sc, pair, spec, mode=1, per_gaussian_shading=True)
    assert np.array_equal(a["img"], b["img"])


@pytest.mark.parametrize("seed", [0, 1])
def test_fd_of_the_per_gaussian_shaded_render(seed):
    sc, pair, spec = _tiny(seed)
    dimg = sg.random_dimg(seed + 80, pair.W * pair.H)
    r = O.render_pair(sc, pair, spec, dimg=dimg, per_gaussian_shading=True)
    r0 = O.render_pair(sc, pair, spec, per_gaussian_shading=True)
    live = np.flatnonzero(r0["rect"][:, 0] <= r0["rect"][:, 1])
    rng = np.random.default_rng(seed)

    def loss():
        q = O.render_pair(sc, pair, spec, per_gaussian_shading=True)
        return float((q["img"] * dimg).sum()), q["ncontrib"].copy(), q["margin"][:, 2].copy()

    _, nc0, cl0 = loss()
    used, bad = 0, []
    for name in PARAMS + ["W0"]:
        for _ in range(4):
            if name == "W0":
                arr, idx = spec.weights[0], (int(rng.integers(spec.weights[0].shape[0])),
                                             int(rng.integers(spec.weights[0].shape[1])))
                ana = r["dW"][0][idx]
            else:
                arr = getattr(sc, name)
                g = int(rng.choice(live))
                idx = (g,) if arr.ndim == 1 else (g, int(rng.integers(arr.shape[1])))
                ana = r["grads"][name][idx]
            x0 = float(arr[idx])
            h = 1e-6 * max(1.0, abs(x0))
            arr[idx] = x0 + h
            lp, ncp, clp = loss()
            arr[idx] = x0 - h
            lm, ncm, clm = loss()
            arr[idx] = x0
            if not (np.array_equal(ncp, nc0) and np.array_equal(ncm, nc0)
                    and np.array_equal(clp, cl0) and np.array_equal(clm, cl0)):
                continue
            fd = (lp - lm) / (2 * h)
            used += 1
            if abs(fd - ana) > 2e-5 * max(abs(fd), abs(ana), 1e-3):
                bad.append((name, idx, fd, ana))
    assert used >= 30, used
    assert not bad, bad[:5]
