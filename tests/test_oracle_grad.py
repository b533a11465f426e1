"""Pin the oracle's hand-derived backward with FP64 central finite differences.

Loss = sum(dimg * image) for a fixed seeded dimg, so d(loss)/d(theta) is the
oracle's analytic gradient. Central differences with h = 1e-6 max(1, |theta|)
in FP64 are independent of that derivation. A sample whose +-h evaluation
changes a discrete decision (which Gaussians contribute at a pixel, or which
contributions are clamped at alpha_max) straddles a jump and is skipped; the
test requires that most samples are usable.
"""
import numpy as np
import pytest

import oracle as O
import scenegen as sg


def _tiny(seed, N=24, kind="basic", widths=(16, 16), log_s_mean=-1.8, res=32, metal_zero=False):
    sc = sg.shell_scene(seed, N)
    rng = np.random.default_rng(seed + 100)
    sc.log_s = sg.f32(rng.normal(log_s_mean, 0.25, (N, 3)))
    sc.normal = sg.f32(sc.normal + rng.normal(0, 0.3, (N, 3)))
    if not metal_zero:
        sc.metal = sg.f32(rng.uniform(0, 1, N))
    sc.vis = sg.f32(rng.uniform(0, 1, N))
    cam = 3.0 * np.array([1.0, 0.2, 1.0]) / np.linalg.norm([1.0, 0.2, 1.0])
    pair = sg._make_pair(cam, [1.5, -2.0, 3.0], res, res)
    spec = sg.mlp_spec(seed + 7, kind, list(widths))
    return sc, pair, spec


def _loss(sc, pair, spec, dimg):
    r = O.render_pair(sc, pair, spec)
    return float((r["img"] * dimg).sum()), r["ncontrib"].copy(), r["margin"][:, 2].copy()


def _fd_check(sc, pair, spec, picks, dimg, rtol=2e-5):
    r = O.render_pair(sc, pair, spec, dimg=dimg)
    _, nc0, cl0 = _loss(sc, pair, spec, dimg)
    used, bad = 0, []
    for name, idx in picks:
        if name[0] in "Wb" and name[1:].isdigit():
            l = int(name[1:])
            arr = (spec.weights if name[0] == "W" else spec.biases)[l]
            ana = (r["dW"] if name[0] == "W" else r["db"])[l][idx]
        else:
            arr = getattr(sc, name)
            ana = r["grads"][name][idx]
        x0 = float(arr[idx])
        h = 1e-6 * max(1.0, abs(x0))
        arr[idx] = x0 + h
        lp, ncp, clp = _loss(sc, pair, spec, dimg)
        arr[idx] = x0 - h
        lm, ncm, clm = _loss(sc, pair, spec, dimg)
        arr[idx] = x0
        if not (np.array_equal(ncp, nc0) and np.array_equal(ncm, nc0)
                and np.array_equal(clp, cl0) and np.array_equal(clm, cl0)):
            continue
        fd = (lp - lm) / (2 * h)
        used += 1
        scale = max(abs(fd), abs(ana), 1e-3)
        if abs(fd - ana) > rtol * scale:
            bad.append((name, idx, fd, ana))
    return used, bad


PARAMS = ["mu", "log_s", "quat", "logit_o", "normal", "base", "rough", "metal", "sss", "vis"]


@pytest.mark.parametrize("seed", [0, 1])
def test_fd_scene_parameters_basic_mlp(seed):
    sc, pair, spec = _tiny(seed)
    dimg = sg.random_dimg(seed + 50, pair.W * pair.H)
    r = O.render_pair(sc, pair, spec)
    live = np.flatnonzero(r["rect"][:, 0] <= r["rect"][:, 1])
    rng = np.random.default_rng(seed)
    picks = []
    for name in PARAMS:
        arr = getattr(sc, name)
        for _ in range(6):
            g = int(rng.choice(live))
            idx = (g,) if arr.ndim == 1 else (g, int(rng.integers(arr.shape[1])))
            picks.append((name, idx))
    used, bad = _fd_check(sc, pair, spec, picks, dimg)
    assert used >= 0.8 * len(picks), used
    assert not bad, bad[:5]


def test_fd_mlp_weights_basic():
    sc, pair, spec = _tiny(3)
    dimg = sg.random_dimg(53, pair.W * pair.H)
    rng = np.random.default_rng(3)
    picks = []
    for l, W in enumerate(spec.weights):
        for _ in range(5):
            picks.append((f"W{l}", (int(rng.integers(W.shape[0])), int(rng.integers(W.shape[1])))))
        picks.append((f"b{l}", (int(rng.integers(W.shape[0])),)))
    used, bad = _fd_check(sc, pair, spec, picks, dimg)
    assert used >= 0.8 * len(picks)
    assert not bad, bad[:5]


def test_fd_pe6_mlp_inputs_and_weights():
    """The Fourier-encoded network of the 300K configuration (FP64 mode)."""
    sc, pair, _ = _tiny(4)
    spec = sg.mlp_spec(9, "pe6", [32, 32])
    dimg = sg.random_dimg(54, pair.W * pair.H)
    r = O.render_pair(sc, pair, spec)
    live = np.flatnonzero(r["rect"][:, 0] <= r["rect"][:, 1])
    rng = np.random.default_rng(4)
    picks = [("mu", (int(rng.choice(live)), int(rng.integers(3)))) for _ in range(10)]
    picks += [("normal", (int(rng.choice(live)), int(rng.integers(3)))) for _ in range(5)]
    picks += [("vis", (int(rng.choice(live)),)) for _ in range(5)]
    picks += [("W0", (int(rng.integers(32)), int(rng.integers(50)))) for _ in range(5)]
    picks += [("W2", (int(rng.integers(4)), int(rng.integers(32)))) for _ in range(4)]
    used, bad = _fd_check(sc, pair, spec, picks, dimg)
    assert used >= 0.8 * len(picks)
    assert not bad, bad[:5]


def test_fd_paper_mlp_inputs_and_weights():
    """The paper's network (Leaky-ReLU trunk, two heads): its inputs include
    the rotation and scale, so quat and log_s gradients combine the projection
    path and the network path."""
    sc, pair, _ = _tiny(6)
    spec = sg.mlp_spec(10, "paper", [])
    dimg = sg.random_dimg(56, pair.W * pair.H)
    r = O.render_pair(sc, pair, spec)
    live = np.flatnonzero(r["rect"][:, 0] <= r["rect"][:, 1])
    rng = np.random.default_rng(6)
    picks = [("mu", (int(rng.choice(live)), int(rng.integers(3)))) for _ in range(6)]
    picks += [("quat", (int(rng.choice(live)), int(rng.integers(4)))) for _ in range(6)]
    picks += [("log_s", (int(rng.choice(live)), int(rng.integers(3)))) for _ in range(6)]
    picks += [("normal", (int(rng.choice(live)), int(rng.integers(3)))) for _ in range(3)]
    picks += [("vis", (int(rng.choice(live)),)) for _ in range(3)]
    picks += [("W0", (int(rng.integers(64)), int(rng.integers(42)))) for _ in range(3)]
    picks += [("W3", (int(rng.integers(32)), int(rng.integers(32)))) for _ in range(3)]
    picks += [("W4", (0, int(rng.integers(32)))) for _ in range(2)]
    picks += [("W5", (int(rng.integers(3)), int(rng.integers(32)))) for _ in range(3)]
    picks += [("b4", (0,)), ("b5", (1,))]
    used, bad = _fd_check(sc, pair, spec, picks, dimg)
    assert used >= 0.8 * len(picks)
    assert not bad, bad[:5]


def test_fd_with_clamped_alpha_and_stop():
    """Dense, opaque Gaussians: alpha clamps at 0.99 and T-stops are common."""
    sc, pair, spec = _tiny(5, N=40, log_s_mean=-1.6)
    sc.logit_o = sg.f32(np.random.default_rng(8).normal(3.0, 2.0, sc.N))
    dimg = sg.random_dimg(55, pair.W * pair.H)
    r = O.render_pair(sc, pair, spec)
    assert r["margin"][:, 2].sum() > 0          # some clamped contributions exist
    live = np.flatnonzero(r["rect"][:, 0] <= r["rect"][:, 1])
    rng = np.random.default_rng(5)
    picks = []
    for name in ["mu", "log_s", "quat", "logit_o", "base", "rough"]:
        arr = getattr(sc, name)
        for _ in range(6):
            g = int(rng.choice(live))
            idx = (g,) if arr.ndim == 1 else (g, int(rng.integers(arr.shape[1])))
            picks.append((name, idx))
    used, bad = _fd_check(sc, pair, spec, picks, dimg)
    assert used >= 0.7 * len(picks)
    assert not bad, bad[:5]


def test_fd_training_objective_of_app_e():
    """The whole training objective of App. E, image loss (0.8 L1 + 0.2 D-SSIM)
    plus the incident-light constraint, through the renderer and the paper's
    network: the gradient that render_pair returns given the image loss's
    dL/dimg and the constraint's dL/dL_in, dL/dv, against central differences
    of the objective. Samples that flip an L1 sign or a clamp of L_in straddle
    a kink and are skipped like the discrete decisions."""
    sc, pair, _ = _tiny(7)
    spec = sg.mlp_spec(11, "paper", [])
    H, W = pair.H, pair.W
    r0 = O.render_pair(sc, pair, spec)
    target = np.clip(r0["img"].reshape(H, W, 3) + np.random.default_rng(70).normal(0, 0.05, (H, W, 3)), 0, 1)

    def objective():
        r = O.render_pair(sc, pair, spec)
        li, _ = O.image_loss(r["img"].reshape(H, W, 3), target)
        lc, _, _ = O.incident_loss(r["Lin"], sc.vis)
        kinks = (np.sign(r["img"].reshape(H, W, 3) - target), np.sign(np.minimum(r["Lin"], 1.0) - sc.vis),
                 r["Lin"] < 1.0)
        return li + lc, r["ncontrib"].copy(), r["margin"][:, 2].copy(), kinks

    _, gimg = O.image_loss(r0["img"].reshape(H, W, 3), target)
    _, dl, dv = O.incident_loss(r0["Lin"], sc.vis)
    r = O.render_pair(sc, pair, spec, dimg=gimg.reshape(-1, 3), dlin_extra=dl, dvis_extra=dv)
    J0, nc0, cl0, k0 = objective()
    live = np.flatnonzero(r["rect"][:, 0] <= r["rect"][:, 1])
    rng = np.random.default_rng(7)
    picks = [("mu", (int(rng.choice(live)), int(rng.integers(3)))) for _ in range(6)]
    picks += [("log_s", (int(rng.choice(live)), int(rng.integers(3)))) for _ in range(4)]
    picks += [("vis", (int(rng.integers(sc.N)),)) for _ in range(6)]
    picks += [("base", (int(rng.choice(live)), int(rng.integers(3)))) for _ in range(3)]
    picks += [("W0", (int(rng.integers(64)), int(rng.integers(42)))) for _ in range(4)]
    picks += [("W4", (0, int(rng.integers(32)))) for _ in range(3)]
    picks += [("b4", (0,)), ("b5", (2,))]
    used, bad = 0, []
    for name, idx in picks:
        if name[0] in "Wb" and name[1:].isdigit():
            l = int(name[1:])
            arr = (spec.weights if name[0] == "W" else spec.biases)[l]
            ana = (r["dW"] if name[0] == "W" else r["db"])[l][idx]
        else:
            arr = getattr(sc, name)
            ana = r["grads"][name][idx]
        x0 = float(arr[idx])
        h = 1e-6 * max(1.0, abs(x0))
        arr[idx] = x0 + h
        Jp, ncp, clp, kp = objective()
        arr[idx] = x0 - h
        Jm, ncm, clm, km = objective()
        arr[idx] = x0
        same = all(np.array_equal(a, b) and np.array_equal(a, c) for a, b, c in zip(k0, kp, km))
        if not (same and np.array_equal(ncp, nc0) and np.array_equal(ncm, nc0)
                and np.array_equal(clp, cl0) and np.array_equal(clm, cl0)):
            continue
        fd = (Jp - Jm) / (2 * h)
        used += 1
        if abs(fd - ana) > 2e-5 * max(abs(fd), abs(ana), 1e-4):
            bad.append((name, idx, fd, ana))
    assert used >= 0.8 * len(picks), used
    assert not bad, bad[:5]
    # the constraint reaches the visibility of Gaussians that no pixel sees
    hidden = np.setdiff1d(np.arange(sc.N), live)
    if hidden.size:
        assert np.allclose(r["grads"]["vis"][hidden], dv[hidden])


def test_fd_config2_size_64_parameters():
    """The analytic backward at a realistic list depth: the 100K-Gaussian blob
    at 512x512 with its 9-64-64-64-4 network, 64 random parameters (36 scene
    parameters of Gaussians that reach the crop, 28 network weights and
    biases with a nonzero gradient). The loss is sum(dimg * image) over a
    56 x 48 pixel crop that holds lit surface, shadow and the silhouette
    (lists of ~60-140 contributions per pixel); only those pixels are
    rendered, which leaves the crop's values exact. v enters neither the
    network nor the shading of this configuration, so it is not sampled."""
    wl = sg.make_workload("c2")
    sc, pair, spec = wl.scenes[0], wl.pairs[0], wl.mlp
    pix = O.all_pixels(pair.W, pair.H)
    crop = pix[(pix[:, 0] >= 112) & (pix[:, 0] < 168) & (pix[:, 1] >= 40) & (pix[:, 1] < 88)].astype(np.int32)
    dimg = sg.random_dimg(5, crop.shape[0])
    r = O.render_pair(sc, pair, spec, pixels=crop, dimg=dimg)
    assert r["ncontrib"].mean() > 50 and r["ncontrib"].max() > 200
    assert 0.5 < (r["ncontrib"] > 0).mean() < 1.0           # silhouette inside the crop

    def loss():
        q = O.render_pair(sc, pair, spec, pixels=crop)
        return float((q["img"] * dimg).sum()), q["ncontrib"].copy(), q["margin"][:, 2].copy()

    _, nc0, cl0 = loss()
    rng = np.random.default_rng(2)
    picks = []
    for name in ["mu", "log_s", "quat", "logit_o", "normal", "base", "rough", "metal", "sss"]:
        gg = r["grads"][name]
        live = np.flatnonzero(np.abs(gg.reshape(gg.shape[0], -1)).sum(1) > 0)
        assert live.size > 100, name
        arr = getattr(sc, name)
        for _ in range(4):
            g = int(rng.choice(live))
            picks.append((name, (g,) if arr.ndim == 1 else (g, int(rng.integers(arr.shape[1])))))
    for l in range(len(spec.weights)):
        for kind, n_pick in (("W", 5), ("b", 2)):
            ana = (r["dW"] if kind == "W" else r["db"])[l]
            nz = np.argwhere(ana != 0)
            for k in rng.choice(len(nz), n_pick, replace=False):
                picks.append((f"{kind}{l}", tuple(int(x) for x in nz[k])))
    assert len(picks) == 64
    used, bad, worst = 0, [], 0.0
    for name, idx in picks:
        if name[0] in "Wb" and name[1:].isdigit():
            l = int(name[1:])
            arr = (spec.weights if name[0] == "W" else spec.biases)[l]
            ana = (r["dW"] if name[0] == "W" else r["db"])[l][idx]
        else:
            arr = getattr(sc, name)
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
            continue                    # a decision flipped inside +-h: a jump, not a derivative
        used += 1
        fd = (lp - lm) / (2 * h)
        rel = abs(fd - ana) / max(abs(fd), abs(ana), 1e-3)
        worst = max(worst, rel)
        if rel > 2e-5:
            bad.append((name, idx, fd, ana))
    assert used >= 56, used
    assert not bad, bad[:5]
