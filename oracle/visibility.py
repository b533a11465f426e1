"""Ray-traced per-Gaussian visibility and the SH visibility term (test
infrastructure only, FP64 numpy; only tests, smoke() and bench's CPU legs use it).

Sec. 3.2 "Incident Light" (and the related-work paragraph on R3DGS): rays are
traced through the Gaussians to estimate each Gaussian's visibility of the
light, and that estimate supervises a learnable per-Gaussian spherical-harmonic
visibility term v; App. E "Losses" weights this ray-traced visibility loss by
lambda_raytrace = 0.01. The paper leaves the tracer's response, the SH degree
and the loss form to R3DGS; the readings taken here:

* visibility of Gaussian i toward the point light l: the transmittance of the
  segment from mu_i to l through every other Gaussian j,
      v_i = prod_j (1 - alpha_j),
  alpha_j = min(alpha_max, o_j exp(-q*/2)) with q* the minimum over the ray of
  the Mahalanobis distance (x - mu_j)^T Sigma_j^-1 (x - mu_j) (the Gaussian's
  peak response along the ray), counted when the peak lies inside the segment
  (0 < t* < |l - mu_i|) and alpha_j >= alpha_min (the compositing rules of
  Eq. 3), Gaussian i itself excluded;
* the SH term: 16 real spherical-harmonic coefficients per Gaussian (degree 3,
  orthonormal basis without the Condon-Shortley phase),
      v_i(w) = clamp(sum_k c_ik Y_k(w), 0, 1),  w = (l - mu_i) / |l - mu_i|;
* the loss per pair: lambda_raytrace * mean over its Gaussians of
  |v_i(w) - v_traced_i| (L1, the traced value a constant target).
"""
from __future__ import annotations

import math

import numpy as np

LAMBDA_RAYTRACE = 0.01
SH_COEFFS = 16

_C0 = 0.5 / math.sqrt(math.pi)
_C1 = math.sqrt(3.0 / (4.0 * math.pi))
_C2a = 0.5 * math.sqrt(15.0 / math.pi)
_C2b = 0.25 * math.sqrt(5.0 / math.pi)
_C2c = 0.25 * math.sqrt(15.0 / math.pi)
_C3a = 0.25 * math.sqrt(35.0 / (2.0 * math.pi))
_C3b = 0.5 * math.sqrt(105.0 / math.pi)
_C3c = 0.25 * math.sqrt(21.0 / (2.0 * math.pi))
_C3d = 0.25 * math.sqrt(7.0 / math.pi)
_C3e = 0.25 * math.sqrt(105.0 / math.pi)


def sh_basis(w):
    """Real SH Y_k(w), k = l^2 + l + m (l <= 3), of unit vectors w (... x 3)."""
    w = np.asarray(w, np.float64)
    x, y, z = w[..., 0], w[..., 1], w[..., 2]
    return np.stack([
        _C0 * np.ones_like(x),
        _C1 * y, _C1 * z, _C1 * x,
        _C2a * x * y, _C2a * y * z, _C2b * (3 * z * z - 1), _C2a * x * z, _C2c * (x * x - y * y),
        _C3a * y * (3 * x * x - y * y), _C3b * x * y * z, _C3c * y * (5 * z * z - 1), _C3d * z * (5 * z * z - 3),
        _C3c * x * (5 * z * z - 1), _C3e * z * (x * x - y * y), _C3a * x * (x * x - 3 * y * y),
    ], axis=-1)


def sh_basis_grad(w):
    """d Y_k / d(x, y, z) of the polynomials above (... x 16 x 3)."""
    w = np.asarray(w, np.float64)
    x, y, z = w[..., 0], w[..., 1], w[..., 2]
    o, zero = np.ones_like(x), np.zeros_like(x)
    rows = [
        (zero, zero, zero),
        (zero, _C1 * o, zero), (zero, zero, _C1 * o), (_C1 * o, zero, zero),
        (_C2a * y, _C2a * x, zero), (zero, _C2a * z, _C2a * y), (zero, zero, _C2b * 6 * z),
        (_C2a * z, zero, _C2a * x), (_C2c * 2 * x, -_C2c * 2 * y, zero),
        (_C3a * 6 * x * y, _C3a * (3 * x * x - 3 * y * y), zero), (_C3b * y * z, _C3b * x * z, _C3b * x * y),
        (zero, _C3c * (5 * z * z - 1), _C3c * 10 * y * z), (zero, zero, _C3d * (15 * z * z - 3)),
        (_C3c * (5 * z * z - 1), zero, _C3c * 10 * x * z), (_C3e * 2 * x * z, -_C3e * 2 * y * z, _C3e * (x * x - y * y)),
        (_C3a * (3 * x * x - 3 * y * y), -_C3a * 6 * x * y, zero),
    ]
    return np.stack([np.stack(r, axis=-1) for r in rows], axis=-2)


def light_dirs(mu, light):
    V = np.asarray(light, np.float64)[None, :] - np.asarray(mu, np.float64)
    r = np.linalg.norm(V, axis=1)
    return V / r[:, None], r


def vis_sh(sh, mu, light):
    """v_i = clamp(c_i . Y(w_i), 0, 1) of one pair's light; returns (v, u) with
    u the unclamped sum."""
    w, _ = light_dirs(mu, light)
    u = np.einsum("nk,nk->n", np.asarray(sh, np.float64), sh_basis(w))
    return np.clip(u, 0.0, 1.0), u


def vis_sh_backward(dv, sh, mu, light):
    """dL/dc and dL/dmu from dL/dv (zero where the clamp is active)."""
    sh = np.asarray(sh, np.float64)
    w, r = light_dirs(mu, light)
    Y = sh_basis(w)
    u = np.einsum("nk,nk->n", sh, Y)
    g = np.asarray(dv, np.float64) * ((u > 0.0) & (u < 1.0))
    dc = g[:, None] * Y
    dw = g[:, None] * np.einsum("nk,nkc->nc", sh, sh_basis_grad(w))
    # w = V / |V|, V = light - mu: dV = (dw - (w . dw) w) / |V|, dmu = -dV
    dV = (dw - np.einsum("nc,nc->n", w, dw)[:, None] * w) / r[:, None]
    return dc, -dV


def rotation(quat):
    """Rotation matrices of (w, x, y, z) quaternions, normalised first."""
    q = np.asarray(quat, np.float64)
    q = q / np.linalg.norm(q, axis=-1, keepdims=True)
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1),
    ], -2)


def trace_visibility(scene, light, alpha_min=1.0 / 255.0, alpha_max=0.99, items=None):
    """Brute-force ray-traced visibility of every Gaussian (or of `items`) of
    `scene` toward `light`. Returns (v, margin) with margin the smallest
    relative distance of any decision (alpha vs alpha_min / alpha_max, the
    peak position vs the segment ends) from its threshold."""
    mu = np.asarray(scene.mu, np.float64)
    N = mu.shape[0]
    R = rotation(scene.quat)                                      # N x 3 x 3
    inv_s = np.exp(-np.asarray(scene.log_s, np.float64))         # N x 3
    o = 1.0 / (1.0 + np.exp(-np.asarray(scene.logit_o, np.float64)))
    light = np.asarray(light, np.float64)
    idx = np.arange(N) if items is None else np.asarray(items)
    v = np.ones(idx.shape[0])
    margin = np.full(idx.shape[0], np.inf)
    for n, i in enumerate(idx):
        seg = light - mu[i]
        tL = np.linalg.norm(seg)
        d = seg / tL
        # local frame of every Gaussian j: x' = S^-1 R^T (x - mu_j)
        op = np.einsum("nji,nj->ni", R, mu[i][None, :] - mu) * inv_s
        dp = np.einsum("nji,j->ni", R, d) * inv_s
        dd = np.einsum("ni,ni->n", dp, dp)
        od = np.einsum("ni,ni->n", op, dp)
        t = -od / dd
        q = np.einsum("ni,ni->n", op, op) - od * od / dd
        a_raw = o * np.exp(-0.5 * np.maximum(q, 0.0))
        a = np.minimum(alpha_max, a_raw)
        take = (t > 0.0) & (t < tL) & (a >= alpha_min)
        take[i] = False
        v[n] = float(np.prod(1.0 - a[take]))
        near = np.ones(N, bool)
        near[i] = False
        m1 = np.abs(a_raw - alpha_min) / alpha_min
        m2 = np.abs(a_raw - alpha_max) / alpha_max
        m3 = np.abs(t) / tL
        m4 = np.abs(t - tL) / tL
        # only decisions that could change the product matter: Gaussians near
        # the alpha threshold, or near a segment end with a visible alpha
        rel = np.minimum(m1, np.where(a >= alpha_min, np.minimum(np.minimum(m3, m4), m2), np.inf))
        margin[n] = float(rel[near].min()) if near.any() else np.inf
    return v, margin


def vis_loss(v, v_traced, lam=LAMBDA_RAYTRACE):
    """lambda * mean |v - v_traced| of one pair and its gradient w.r.t. v."""
    d = np.asarray(v, np.float64) - np.asarray(v_traced, np.float64)
    return lam * float(np.abs(d).mean()), lam * np.sign(d) / d.size
