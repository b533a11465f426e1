"""Training losses of App. E "Losses" (test infrastructure only, FP64 numpy;
only tests, smoke() and bench's CPU legs use it).

Image loss per view/light pair (App. E: "as in 3D GS"):
    L_img = (1 - lambda_dssim) L1 + lambda_dssim (1 - SSIM),  lambda_dssim = 0.2
with L1 the mean absolute difference over the pair's pixels and channels and
SSIM the structural similarity of Wang et al. (2004) averaged over pixels and
channels: per channel, local means, variances and covariance under an 11 x 11
Gaussian window (sigma 1.5, normalised, zero padding outside the image),
    S = (2 mu_x mu_y + C1)(2 s_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(s_x^2 + s_y^2 + C2)),
C1 = 0.01^2, C2 = 0.03^2. The gradient follows the definition by the chain
rule through the windowed moments.

Incident-light constraint per pair (App. E: the clamped predicted incident
light is kept close to the visibility by an L1 loss, lambda = 0.02):
    L_inc = lambda_inc * mean over the pair's Gaussians of |min(L_in, 1) - v|.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.ndimage as nd

SSIM_WIN = 11
SSIM_SIGMA = 1.5
SSIM_C1 = 0.01 ** 2
SSIM_C2 = 0.03 ** 2
LAMBDA_DSSIM = 0.2
LAMBDA_INCIDENT = 0.02


def gaussian_window(size=SSIM_WIN, sigma=SSIM_SIGMA):
    """Normalised 1-D Gaussian taps (the 2-D window is their outer product)."""
    r = np.arange(size) - (size - 1) / 2.0
    w = np.exp(-r ** 2 / (2.0 * sigma ** 2))
    return w / w.sum()


def window_mean(a):
    """Windowed mean of an H x W (x C) array, zero outside the image."""
    w = gaussian_window()
    a = nd.correlate1d(np.asarray(a, np.float64), w, axis=0, mode="constant", cval=0.0)
    return nd.correlate1d(a, w, axis=1, mode="constant", cval=0.0)


def ssim_map(x, y):
    """Per-pixel, per-channel SSIM of images x, y (H x W x 3)."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    mx, my = window_mean(x), window_mean(y)
    sxx = window_mean(x * x) - mx * mx
    syy = window_mean(y * y) - my * my
    sxy = window_mean(x * y) - mx * my
    return ((2 * mx * my + SSIM_C1) * (2 * sxy + SSIM_C2)) / ((mx * mx + my * my + SSIM_C1) * (sxx + syy + SSIM_C2))


def ssim(x, y):
    """Mean SSIM of images x, y (H x W x 3) and its gradient w.r.t. x."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    mx, my = window_mean(x), window_mean(y)
    sxx = window_mean(x * x) - mx * mx
    syy = window_mean(y * y) - my * my
    sxy = window_mean(x * y) - mx * my
    A1, A2 = 2 * mx * my + SSIM_C1, 2 * sxy + SSIM_C2
    B1, B2 = mx * mx + my * my + SSIM_C1, sxx + syy + SSIM_C2
    S = (A1 * A2) / (B1 * B2)
    n = S.size
    # dS/d(moments) at every pixel, for the mean over n values
    dS_dA1, dS_dA2 = A2 / (B1 * B2) / n, A1 / (B1 * B2) / n
    dS_dB1, dS_dB2 = -S / B1 / n, -S / B2 / n
    d_mx = dS_dA1 * 2 * my + dS_dB1 * 2 * mx        # through mu_x (direct)
    d_sxx = dS_dB2                                  # through s_x^2 = E[x^2] - mu_x^2
    d_sxy = dS_dA2 * 2                              # through s_xy = E[xy] - mu_x mu_y
    d_mx = d_mx - 2 * mx * d_sxx - my * d_sxy       # moments -> (mu_x, E[x^2], E[xy])
    # the window is symmetric, so its adjoint is the same windowed sum
    g = window_mean(d_mx) + 2 * x * window_mean(d_sxx) + y * window_mean(d_sxy)
    return float(S.mean()), g


def image_loss(img, target, lam=LAMBDA_DSSIM):
    """L_img of one pair (images H x W x 3) and dL_img / d img."""
    img = np.asarray(img, np.float64)
    target = np.asarray(target, np.float64)
    d = img - target
    l1 = float(np.abs(d).mean())
    s, gs = ssim(img, target)
    loss = (1.0 - lam) * l1 + lam * (1.0 - s)
    grad = (1.0 - lam) * np.sign(d) / d.size - lam * gs
    return loss, grad


def incident_loss(L_in, vis, lam=LAMBDA_INCIDENT):
    """L_inc of one pair and its gradients w.r.t. L_in and v."""
    L_in = np.asarray(L_in, np.float64)
    vis = np.asarray(vis, np.float64)
    c = np.minimum(L_in, 1.0)
    d = c - vis
    n = L_in.size
    loss = lam * float(np.abs(d).mean())
    s = lam * np.sign(d) / n
    return loss, s * (L_in < 1.0), -s
