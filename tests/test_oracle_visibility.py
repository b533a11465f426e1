"""Pins of the oracle's ray-traced visibility and SH visibility term
(oracle/visibility.py) against library routines, closed forms and brute force."""
import math
from dataclasses import replace

import numpy as np
import pytest
import scipy.special as sp

import oracle as O
import oracle.visibility as V
import scenegen as sg


def _scipy_real_sh(l, m, w):
    th = np.arccos(np.clip(w[:, 2], -1, 1))
    ph = np.arctan2(w[:, 1], w[:, 0])
    if m == 0:
        return np.real(sp.sph_harm_y(l, 0, th, ph))
    Y = sp.sph_harm_y(l, abs(m), th, ph)
    return math.sqrt(2.0) * (-1) ** m * (np.real(Y) if m > 0 else np.imag(Y))


def _unit(rng, n):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def test_sh_basis_equals_scipy_real_harmonics():
    w = _unit(np.random.default_rng(0), 200)
    Y = V.sh_basis(w)
    k = 0
    for l in range(4):
        for m in range(-l, l + 1):
            np.testing.assert_allclose(Y[:, k], _scipy_real_sh(l, m, w), atol=1e-12)
            k += 1


def test_sh_basis_orthonormal_by_quadrature():
    xg, wg = np.polynomial.legendre.leggauss(24)          # exact for the degree-6 products in cos(theta)
    ph = (np.arange(48) + 0.5) * 2 * np.pi / 48
    ct, pp = np.meshgrid(xg, ph, indexing="ij")
    st = np.sqrt(1 - ct * ct)
    w = np.stack([st * np.cos(pp), st * np.sin(pp), ct], -1).reshape(-1, 3)
    wt = (wg[:, None] * np.full(48, 2 * np.pi / 48)[None, :]).reshape(-1)
    Y = V.sh_basis(w)
    G = np.einsum("n,nk,nj->kj", wt, Y, Y)
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_sh_gradient_equals_finite_differences():
    w = np.random.default_rng(1).normal(size=(20, 3))     # the polynomials, anywhere in R^3
    g = V.sh_basis_grad(w)
    h = 1e-6
    for c in range(3):
        e = np.zeros(3)
        e[c] = h
        fd = (V.sh_basis(w + e) - V.sh_basis(w - e)) / (2 * h)
        np.testing.assert_allclose(g[..., c], fd, atol=1e-7)


def test_vis_sh_equals_clamped_expansion_in_scipy_harmonics():
    """v = clamp(sum_k c_k Y_k(w), 0, 1) with w the unit direction to the
    light and Y_k from scipy; coefficients large enough that both clamps act."""
    rng = np.random.default_rng(6)
    n = 300
    mu = rng.normal(0, 0.5, (n, 3))
    light = np.array([0.5, 1.0, 3.0])
    sh = rng.normal(0, 0.8, (n, 16))
    v, u = V.vis_sh(sh, mu, light)
    w = (light[None, :] - mu) / np.linalg.norm(light[None, :] - mu, axis=1, keepdims=True)
    Y = np.stack([_scipy_real_sh(l, m, w) for l in range(4) for m in range(-l, l + 1)], axis=1)
    ref = np.einsum("nk,nk->n", sh, Y)
    np.testing.assert_allclose(u, ref, atol=1e-12)
    np.testing.assert_allclose(v, np.clip(ref, 0.0, 1.0), atol=1e-12)
    assert (ref < 0).sum() > 20 and (ref > 1).sum() > 20


def test_vis_sh_backward_equals_finite_differences():
    rng = np.random.default_rng(2)
    n = 12
    mu = rng.normal(0, 0.5, (n, 3))
    light = np.array([1.5, -2.0, 3.0])
    sh = rng.normal(0, 0.3, (n, 16))
    sh[:, 0] += 1.0                                      # v mostly inside (0, 1)
    dv = rng.uniform(-1, 1, n)
    v, u = V.vis_sh(sh, mu, light)
    inside = (u > 1e-3) & (u < 1 - 1e-3)
    assert inside.sum() >= n // 2
    dc, dmu = V.vis_sh_backward(dv, sh, mu, light)
    h = 1e-6
    f = lambda s, m: float((V.vis_sh(s, m, light)[0] * dv).sum())
    for i in np.flatnonzero(inside)[:5]:
        for k in (0, 3, 7, 15):
            sp_, sm_ = sh.copy(), sh.copy()
            sp_[i, k] += h
            sm_[i, k] -= h
            assert abs((f(sp_, mu) - f(sm_, mu)) / (2 * h) - dc[i, k]) < 1e-6
        for c in range(3):
            mp, mm = mu.copy(), mu.copy()
            mp[i, c] += h
            mm[i, c] -= h
            assert abs((f(sh, mp) - f(sh, mm)) / (2 * h) - dmu[i, c]) < 1e-6
    assert np.all(dc[~((u > 0) & (u < 1))] == 0)


def test_rotation_scale_reproduce_the_covariance():
    sc = sg.shell_scene(3, 16)
    R = V.rotation(sc.quat)
    S2 = np.exp(2 * np.asarray(sc.log_s, np.float64))
    for g in range(sc.N):
        Sig = R[g] @ np.diag(S2[g]) @ R[g].T
        np.testing.assert_allclose(Sig, O.covariance(sc.log_s[g], sc.quat[g]), rtol=1e-12, atol=1e-15)


def _scene(mu, log_s, quat, logit_o):
    n = len(mu)
    base = sg.shell_scene(0, n)
    return replace(base, mu=np.asarray(mu, np.float64), log_s=np.asarray(log_s, np.float64),
                   quat=np.asarray(quat, np.float64), logit_o=np.asarray(logit_o, np.float64))


def _logit(o):
    return math.log(o / (1 - o))


def test_trace_closed_forms():
    light = np.array([0.0, 0.0, 4.0])
    I = [1.0, 0.0, 0.0, 0.0]
    s = math.log(0.1)
    # Gaussian 0 at the origin; occluder 1 on the segment (peak on the ray,
    # q* = 0, alpha = o); occluder 2 off the ray by r = 0.15 (alpha = o exp(-r^2 / 2 s^2));
    # 3 behind the origin and 4 beyond the light (peaks outside the segment)
    o1, o2 = 0.6, 0.7
    sc = _scene([[0, 0, 0], [0, 0, 2.0], [0.15, 0, 1.0], [0, 0, -1.0], [0, 0, 5.0]],
                [[s, s, s]] * 5, [I] * 5, [_logit(0.5), _logit(o1), _logit(o2), _logit(0.9), _logit(0.9)])
    v, _ = V.trace_visibility(sc, light, items=[0])
    a2 = o2 * math.exp(-0.5 * (0.15 / 0.1) ** 2)
    assert abs(v[0] - (1 - o1) * (1 - a2)) < 1e-12
    # alpha clamps at 0.99; a far-off Gaussian (alpha < 1/255) does not count
    sc2 = _scene([[0, 0, 0], [0, 0, 2.0], [1.0, 0, 2.0]], [[s, s, s]] * 3, [I] * 3,
                 [0.0, _logit(0.999), _logit(0.99)])
    v2, _ = V.trace_visibility(sc2, light, items=[0])
    assert abs(v2[0] - 0.01) < 1e-12
    # nothing in the way
    v3, _ = V.trace_visibility(sc, light, items=[3])     # from behind: 0, 1, 2 lie on its segment
    v4, _ = V.trace_visibility(sc, light, items=[4])     # beyond the light: nothing
    assert v4[0] == 1.0 and v3[0] < 1.0


def test_trace_peak_response_equals_dense_ray_sampling():
    """q* (the closed-form minimum over the ray) against a dense sampling of
    the Mahalanobis distance along the segment, for rotated anisotropic
    occluders."""
    rng = np.random.default_rng(4)
    n = 6
    mu = np.concatenate([[[0, 0, 0]], rng.uniform(-0.3, 0.3, (n, 3)) + [0, 0, 1.5]])
    log_s = np.concatenate([[[-3, -3, -3]], rng.normal(-1.8, 0.4, (n, 3))])
    quat = np.concatenate([[[1, 0, 0, 0]], rng.normal(size=(n, 4))])
    sc = _scene(mu, log_s, quat, [0.0] + [_logit(0.8)] * n)
    light = np.array([0.2, -0.1, 4.0])
    v, _ = V.trace_visibility(sc, light, items=[0])
    R = V.rotation(quat)
    t = np.linspace(0, np.linalg.norm(light), 400001)[1:-1]
    d = light / np.linalg.norm(light)
    X = t[:, None] * d[None, :]
    prod = 1.0
    for j in range(1, n + 1):
        Sinv = R[j] @ np.diag(np.exp(-2 * log_s[j])) @ R[j].T
        D = X - mu[j]
        q = np.einsum("ti,ij,tj->t", D, Sinv, D)
        k = int(np.argmin(q))
        if 0 < k < len(t) - 1:                            # peak inside the segment
            a = min(0.99, 0.8 * math.exp(-0.5 * q[k]))
            if a >= 1 / 255:
                prod *= 1 - a
    assert abs(v[0] - prod) < 1e-6


def test_vis_loss_gradient():
    rng = np.random.default_rng(5)
    v, vt = rng.uniform(0, 1, 50), rng.uniform(0, 1, 50)
    L, g = V.vis_loss(v, vt)
    assert abs(L - 0.01 * np.abs(v - vt).mean()) < 1e-15
    h = 1e-7
    for i in range(5):
        e = np.zeros(50)
        e[i] = h
        assert abs((V.vis_loss(v + e, vt)[0] - V.vis_loss(v - e, vt)[0]) / (2 * h) - g[i]) < 1e-9
