"""FP64 CPU oracle for the SSS Gaussian-splatting OLAT render.

TEST INFRASTRUCTURE ONLY: only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference legs may import this package. It shares no code with
the CUDA path (paper_2408_12282_gb300) and never imports it.

Contents
  * the raster stages (EWA projection, Eq. 2; alpha compositing, Eq. 3;
    deferred Disney/Cook-Torrance shading, Eq. 4, blended with the SSS
    residual, Eq. 7; and their hand-derived backward) in plain C, FP64
    (sssgs_oracle.c, loaded through ctypes);
  * the joint SSS / incident-light MLP f_Theta of Eq. 6 with the Fourier
    encoding of the mean (Section 3.2 "SSS Modeling", Appendix E "Network"),
    in numpy FP64, with an optional BF16-emulating mode (inputs, weights and
    each layer's activations rounded to bfloat16 round-to-nearest-even,
    accumulation in FP64);
  * a plain stable sort for tile binning (orc_bin).

Parity pins live in tests/test_oracle_*.py (closed forms, invariants, brute
force, finite differences, an independent torch-autograd restatement).
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass

import numpy as np

from . import build as _build
from .losses import image_loss, incident_loss, ssim, ssim_map  # noqa: F401  (training losses)

__all__ = ["Cfg", "lib", "render_pair", "render_workload_pair", "mlp_inputs",
           "mlp_forward", "mlp_backward", "input_grads", "brdf", "bin_sort",
           "project", "bf16_round", "cam_array", "DEFAULT_CFG"]

_LIB = None
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_up = ctypes.POINTER(ctypes.c_uint32)


def lib():
    """Load (building if needed) the C oracle."""
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.orc_project.argtypes = [ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _ip, _up]
        L.orc_render.argtypes = [ctypes.c_int, _dp, _ip, _up, _dp, _dp, _dp, _dp,
                                 ctypes.c_int, ctypes.c_int, _ip, _dp, _dp, _ip, _dp,
                                 _dp, _dp, _dp]
        L.orc_project_bwd.argtypes = [ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp, _ip,
                                      _dp, _dp, _dp, _dp, _dp, _dp]
        L.orc_brdf.argtypes = [_dp, _dp, _dp, _dp, ctypes.c_double, ctypes.c_double, _dp, _dp]
        L.orc_shade.argtypes = [ctypes.c_int, _dp, _ip, _ip, _dp, _dp, _dp, _dp, _dp, _dp]
        L.orc_bin.argtypes = [ctypes.c_int, _ip, _ip, _up, _ip, _ip, ctypes.c_int,
                              ctypes.c_longlong, _up, _up, _up]
        L.orc_bin.restype = ctypes.c_longlong
        L.orc_covariance.argtypes = [_dp, _dp, _dp]
        _LIB = L
    return _LIB


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(_ip)


def _u(a):
    a = np.ascontiguousarray(a, dtype=np.uint32)
    return a, a.ctypes.data_as(_up)


def _f32(x):
    return float(np.float32(x))


@dataclass
class Cfg:
    """Render conventions (float32-representable values, shared by both sides)."""
    tile: int = 16
    dilation: float = _f32(0.3)
    det_eps: float = _f32(1e-6)
    z_near: float = _f32(0.2)
    alpha_min: float = _f32(1.0 / 255.0)
    alpha_max: float = _f32(0.99)
    T_min: float = _f32(1e-4)
    A_eps: float = _f32(1e-6)

    def array(self):
        return np.array([self.tile, self.dilation, self.det_eps, self.z_near,
                         self.alpha_min, self.alpha_max, self.T_min, self.A_eps])


DEFAULT_CFG = Cfg()


def cam_array(pair) -> np.ndarray:
    return np.concatenate([np.asarray(pair.R, np.float64).ravel(), np.asarray(pair.t, np.float64),
                           [pair.fx, pair.fy, pair.cx, pair.cy, pair.W, pair.H]])


# ----------------------------------------------------------------------------
# MLP (Eq. 6), numpy FP64
# ----------------------------------------------------------------------------

def bf16_round(x):
    """Round to bfloat16 (8 significant bits), round-to-nearest-even, in FP64."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)                      # x = m 2^e, |m| in [0.5, 1)
    return np.ldexp(np.rint(np.ldexp(m, 8)), e - 8)


def _normalize(v):
    n = np.linalg.norm(v, axis=1, keepdims=True)
    return v / n, n


LRELU_SLOPE = 0.01      # Leaky-ReLU negative slope of the paper's network (not stated; PyTorch default)


def mlp_inputs(kind, mu, normal, vis, cam_center, light, quat=None, log_s=None):
    """Per-Gaussian network input for one view/light pair.

    basic: [mu, w_out, w_in] (9)
    pe6:   [sin(2^k pi mu), cos(2^k pi mu) for k < 6 (36), mu (3), w_out (3),
            w_in (3), n (3), |light - mu| (1), v (1)] = 50, zero-padded to 64.
    paper: [n (3), unit(q) (4), exp(log_s) (3), w_in (3), w_out (3),
            |light - mu| (1), v (1), sin(2^k pi mu), cos(2^k pi mu) for k < 4
            (24)] = 42, zero-padded to 48 (App. E "Network").
    w_out = unit(camera - mu), w_in = unit(light - mu).
    """
    wo, _ = _normalize(np.asarray(cam_center)[None, :] - mu)
    wi, dl = _normalize(np.asarray(light)[None, :] - mu)
    if kind == "basic":
        return np.concatenate([mu, wo, wi], axis=1)
    if kind == "paper":
        qn, _ = _normalize(np.asarray(quat, np.float64))
        feats = [normal, qn, np.exp(log_s), wi, wo, dl, vis[:, None]]
        for k in range(4):
            feats.append(np.sin((2.0 ** k) * math.pi * mu))
            feats.append(np.cos((2.0 ** k) * math.pi * mu))
        X = np.concatenate(feats, axis=1)
        return np.concatenate([X, np.zeros((X.shape[0], 6))], axis=1)
    feats = []
    for k in range(6):
        feats.append(np.sin((2.0 ** k) * math.pi * mu))
        feats.append(np.cos((2.0 ** k) * math.pi * mu))
    X = np.concatenate(feats + [mu, wo, wi, normal, dl, vis[:, None]], axis=1)
    return np.concatenate([X, np.zeros((X.shape[0], 14))], axis=1)


def _lrelu(z):
    return np.where(z > 0, z, LRELU_SLOPE * z)


def _dlrelu(a):
    """Leaky-ReLU derivative from the activation (same sign as the input)."""
    return np.where(a > 0, 1.0, LRELU_SLOPE)


def mlp_forward(spec, X, bf16=False):
    """basic / pe6: Linear/ReLU chain; heads: sigmoid -> L_SSS (3), ReLU -> L_in (1).
    paper: trunk of three Linear + Leaky-ReLU layers (W0..W2); incident head
    Linear + Leaky-ReLU (W3) then Linear + ReLU -> L_in (W4); SSS head
    Linear + sigmoid -> L_SSS (W5), both on the trunk output. Returns the
    layer inputs `acts`, the head pre-activations y = [SSS (3), incident (1)]
    and the outputs."""
    rnd = bf16_round if bf16 else (lambda a: a)
    if spec.kind == "paper":
        W = [rnd(np.asarray(w, np.float64)) for w in spec.weights]
        b = [np.asarray(v, np.float64) for v in spec.biases]
        h = rnd(X)
        acts = [h]
        for l in range(3):
            h = rnd(_lrelu(h @ W[l].T + b[l]))
            acts.append(h)
        t = h
        hid = rnd(_lrelu(t @ W[3].T + b[3]))
        acts.append(hid)
        zi = hid @ W[4].T + b[4]
        zs = t @ W[5].T + b[5]
        y = np.concatenate([zs, zi], axis=1)
        Ls = 1.0 / (1.0 + np.exp(-y[:, :3]))
        Lin = np.maximum(y[:, 3], 0.0)
        return acts, y, Ls, Lin
    h = rnd(X)
    acts = [h]
    nl = len(spec.weights)
    y = None
    for l in range(nl):
        W = rnd(np.asarray(spec.weights[l], np.float64))
        z = h @ W.T + np.asarray(spec.biases[l], np.float64)
        if l < nl - 1:
            h = rnd(np.maximum(z, 0.0))
            acts.append(h)
        else:
            y = z
    Ls = 1.0 / (1.0 + np.exp(-y[:, :3]))
    Lin = np.maximum(y[:, 3], 0.0)
    return acts, y, Ls, Lin


def mlp_backward(spec, acts, y, Ls, dLs, dLin, bf16=False):
    """Backward of mlp_forward. Returns (dW list, db list, dX).

    BF16 mode rounds each layer's pre-activation gradient dz to bfloat16
    before it is used: as a GEMM operand (dW = dz^T h, dh = dz W) and in the
    bias gradient db = sum over rows of dz, i.e. every use of dz sees the same
    bf16 value, as when dz is stored in bf16 once."""
    rnd = bf16_round if bf16 else (lambda a: a)
    if spec.kind == "paper":
        return _paper_backward(spec, acts, y, Ls, dLs, dLin, rnd)
    nl = len(spec.weights)
    dz = np.zeros_like(y)
    dz[:, :3] = dLs * Ls * (1.0 - Ls)
    dz[:, 3] = dLin * (y[:, 3] > 0)
    dWs = [None] * nl
    dbs = [None] * nl
    for l in range(nl - 1, -1, -1):
        W = rnd(np.asarray(spec.weights[l], np.float64))
        dzr = rnd(dz)
        dWs[l] = dzr.T @ acts[l]
        dbs[l] = dzr.sum(axis=0)
        dh = dzr @ W
        if l > 0:
            dz = dh * (acts[l] > 0)
        else:
            dX = dh
    return dWs, dbs, dX


def _paper_backward(spec, acts, y, Ls, dLs, dLin, rnd):
    """Backward of the paper network (same bf16 convention as the chain:
    every pre-activation gradient is rounded once and used everywhere)."""
    W = [rnd(np.asarray(w, np.float64)) for w in spec.weights]
    X, h1, h2, t, hid = acts
    dWs, dbs = [None] * 6, [None] * 6
    dzs = rnd(dLs * Ls * (1.0 - Ls))                       # SSS head
    dzi = rnd((dLin * (y[:, 3] > 0))[:, None])              # incident output
    dWs[5], dbs[5] = dzs.T @ t, dzs.sum(axis=0)
    dWs[4], dbs[4] = dzi.T @ hid, dzi.sum(axis=0)
    dzh = rnd((dzi @ W[4]) * _dlrelu(hid))                 # incident hidden
    dWs[3], dbs[3] = dzh.T @ t, dzh.sum(axis=0)
    dt = dzs @ W[5] + dzh @ W[3]
    hs = [X, h1, h2, t]
    dz = rnd(dt * _dlrelu(t))
    for l in range(2, -1, -1):
        dWs[l], dbs[l] = dz.T @ hs[l], dz.sum(axis=0)
        dh = dz @ W[l]
        if l > 0:
            dz = rnd(dh * _dlrelu(hs[l]))
        else:
            dX = dh
    return dWs, dbs, dX


def input_grads(kind, dX, mu, cam_center, light, quat=None, log_s=None):
    """Map dLoss/dX to (dmu, dn, dv) through the input encoding; for the
    paper network also (dquat, dlog_s): (dmu, dn, dv, dq, dls)."""
    Vo = np.asarray(cam_center)[None, :] - mu
    Vi = np.asarray(light)[None, :] - mu
    wo, lo = _normalize(Vo)
    wi, li = _normalize(Vi)

    def back_unit(w, l, g):            # d/dmu of unit(P - mu) applied to g
        return -(g - w * np.sum(w * g, axis=1, keepdims=True)) / l

    if kind == "basic":
        dmu = dX[:, 0:3] + back_unit(wo, lo, dX[:, 3:6]) + back_unit(wi, li, dX[:, 6:9])
        return dmu, np.zeros_like(mu), np.zeros(mu.shape[0])
    if kind == "paper":
        q = np.asarray(quat, np.float64)
        qn, ql = _normalize(q)
        gq = dX[:, 3:7]
        dq = (gq - qn * np.sum(qn * gq, axis=1, keepdims=True)) / ql
        dls = dX[:, 7:10] * np.exp(log_s)
        dmu = back_unit(wi, li, dX[:, 10:13]) + back_unit(wo, lo, dX[:, 13:16]) - dX[:, 16:17] * wi
        col = 18
        for k in range(4):
            f = (2.0 ** k) * math.pi
            dmu += dX[:, col:col + 3] * f * np.cos(f * mu)
            col += 3
            dmu -= dX[:, col:col + 3] * f * np.sin(f * mu)
            col += 3
        return dmu, dX[:, 0:3].copy(), dX[:, 17].copy(), dq, dls
    dmu = np.zeros_like(mu)
    col = 0
    for k in range(6):
        f = (2.0 ** k) * math.pi
        dmu += dX[:, col:col + 3] * f * np.cos(f * mu)
        col += 3
        dmu -= dX[:, col:col + 3] * f * np.sin(f * mu)
        col += 3
    dmu += dX[:, 36:39]
    dmu += back_unit(wo, lo, dX[:, 39:42])
    dmu += back_unit(wi, li, dX[:, 42:45])
    dn = dX[:, 45:48].copy()
    dmu += dX[:, 48:49] * (-wi)
    dv = dX[:, 49].copy()
    return dmu, dn, dv


# ----------------------------------------------------------------------------
# raster stages
# ----------------------------------------------------------------------------

def project(scene, pair, cfg=DEFAULT_CFG):
    N = scene.N
    proj = np.zeros((N, 16))
    rect = np.zeros((N, 4), np.int32)
    dkey = np.zeros(N, np.uint32)
    a = [_d(scene.mu), _d(scene.log_s), _d(scene.quat), _d(scene.logit_o),
         _d(cam_array(pair)), _d(cfg.array())]
    lib().orc_project(N, *[p for _, p in a], proj.ctypes.data_as(_dp),
                      rect.ctypes.data_as(_ip), dkey.ctypes.data_as(_up))
    return proj, rect, dkey


def all_pixels(W, H):
    jj, ii = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    return np.stack([ii.ravel(), jj.ravel()], axis=1).astype(np.int32)


def gaussian_colors(normal, base, rough, metal, sss, Ls, Lin, mu, cam_center, light, grad_out=None):
    """Per-Gaussian shading (the paper's "w/o Deferred" ablation, App. "Ablation"):
    each Gaussian's colour from its own attributes at its own mean x = mu,
    with the BRDF of Eq. 4 (GGX D, Schlick F, separable Smith V) and the blend
    of Eq. 7:  c = sss L_SSS + (1 - sss) (f_s + f_d) L_in max(n . w_i, 0),
    w_o = unit(camera - x), w_i = unit(light - x), n normalised. Plain PyTorch
    FP64; with grad_out (N x 3) also returns the gradients (autograd) of
    sum(grad_out * c) w.r.t. (normal, base, rough, metal, sss, Ls, Lin, mu)."""
    import torch
    t = lambda a: torch.tensor(np.asarray(a, np.float64), dtype=torch.float64, requires_grad=grad_out is not None)
    n, b, r, m, s, ls, li, x = (t(normal), t(base), t(rough), t(metal), t(sss), t(Ls), t(Lin), t(mu))
    C = torch.tensor(np.asarray(cam_center, np.float64), dtype=torch.float64)
    Lp = torch.tensor(np.asarray(light, np.float64), dtype=torch.float64)
    unit = lambda v, eps=0.0: v / torch.clamp(torch.linalg.norm(v, dim=1, keepdim=True), min=eps)
    wo, wi = unit(C[None, :] - x), unit(Lp[None, :] - x)
    nh = unit(n, 1e-12)
    h = unit(wo + wi, 1e-12)
    dot = lambda a, c: (a * c).sum(dim=1)
    no, ni = torch.clamp(dot(nh, wo), min=0), torch.clamp(dot(nh, wi), min=0)
    nhc, vh = torch.clamp(dot(nh, h), min=0), torch.clamp(dot(wo, h), min=0)
    a2 = (r * r) ** 2
    den = nhc * nhc * (a2 - 1) + 1
    D = a2 / (math.pi * den * den)
    V = 1.0 / ((no + torch.sqrt(a2 + (1 - a2) * no * no)) * (ni + torch.sqrt(a2 + (1 - a2) * ni * ni)))
    F0 = 0.04 * (1 - m[:, None]) + b * m[:, None]
    Fr = F0 + (1 - F0) * ((1 - vh) ** 5)[:, None]
    fs = D[:, None] * Fr * V[:, None]
    fd = (1 - m[:, None]) * b / math.pi
    c = s[:, None] * ls + (1 - s[:, None]) * (fs + fd) * (li * ni)[:, None]
    if grad_out is None:
        return c.detach().numpy()
    (c * torch.tensor(np.asarray(grad_out, np.float64), dtype=torch.float64)).sum().backward()
    return c.detach().numpy(), tuple(v.grad.numpy() for v in (n, b, r, m, s, ls, li, x))


def render_pair(scene, pair, spec, cfg=DEFAULT_CFG, mode=1, pixels=None, dimg=None,
                bf16=False, mlp_out=None, dlin_extra=None, dvis_extra=None, per_gaussian_shading=False):
    """Forward (and, if dimg is given, backward) of one view/light pair.

    pixels: (P x 2) int array of (i, j) to evaluate; default all, row-major.
    dimg:   (P x 3) upstream gradient on those pixels' image values.
    Returns a dict with gbuf (P x 16), img (P x 3), ncontrib, margin (P x 3),
    the per-Gaussian MLP output, and, with dimg, gradients of every parameter
    and of the MLP weights.
    dlin_extra, dvis_extra (N): gradients of further loss terms on the
    predicted incident light L_in and the visibility v of each Gaussian (the
    incident-light constraint of App. E), added before the network backward.
    per_gaussian_shading: shade each Gaussian (gaussian_colors) and composite
    the colours instead of the deferred per-pixel shading."""
    L = lib()
    N = scene.N
    C = pair.center
    kind = spec.kind
    X = mlp_inputs(kind, scene.mu, scene.normal, scene.vis, C, pair.light, scene.quat, scene.log_s)
    acts, y, Ls, Lin = mlp_forward(spec, X, bf16=bf16)
    if mlp_out is not None:      # external network output (tests of the raster alone)
        Ls, Lin = mlp_out[:, :3], mlp_out[:, 3]
    proj, rect, dkey = project(scene, pair, cfg)
    feat = np.concatenate([proj[:, 6:7], scene.normal, scene.base, scene.rough[:, None],
                           scene.metal[:, None], scene.sss[:, None], Ls, Lin[:, None],
                           scene.vis[:, None]], axis=1)
    if per_gaussian_shading:
        colors = gaussian_colors(scene.normal, scene.base, scene.rough, scene.metal, scene.sss, Ls, Lin,
                                 scene.mu, C, pair.light)
        feat = np.concatenate([colors, np.zeros((N, 12))], axis=1)
        mode = mode | 2
    if pixels is None:
        pixels = all_pixels(pair.W, pair.H)
    P = pixels.shape[0]
    gbuf = np.zeros((P, 16))
    img = np.zeros((P, 3))
    nc = np.zeros(P, np.int32)
    margin = np.zeros((P, 3))
    dgeom = np.zeros((N, 6))
    dfeat = np.zeros((N, 15))
    keep = [_d(proj), _i(rect), _u(dkey), _d(feat), _d(cam_array(pair)),
            _d(np.asarray(pair.light, np.float64)), _d(cfg.array()), _i(pixels)]
    if dimg is not None:
        dimg_a, dimg_p = _d(dimg)
    else:
        dimg_p = None
    L.orc_render(N, keep[0][1], keep[1][1], keep[2][1], keep[3][1], keep[4][1], keep[5][1],
                 keep[6][1], int(mode), P, keep[7][1], gbuf.ctypes.data_as(_dp),
                 img.ctypes.data_as(_dp), nc.ctypes.data_as(_ip), margin.ctypes.data_as(_dp),
                 dimg_p, dgeom.ctypes.data_as(_dp), dfeat.ctypes.data_as(_dp))
    out = dict(gbuf=gbuf, img=img, ncontrib=nc, margin=margin, proj=proj, rect=rect,
               dkey=dkey, Ls=Ls, Lin=Lin, feat=feat, pixels=pixels)
    if dimg is None:
        return out
    g = {k: np.zeros_like(v) for k, v in scene.arrays().items()}
    if per_gaussian_shading:          # the composited colours' gradient through each Gaussian's shading
        _, gs = gaussian_colors(scene.normal, scene.base, scene.rough, scene.metal, scene.sss, Ls, Lin,
                                scene.mu, C, pair.light, grad_out=dfeat[:, 0:3])
        dfeat = np.zeros_like(dfeat)  # feature layout of the deferred path (depth unused here)
        dfeat[:, 1:4], dfeat[:, 4:7], dfeat[:, 7], dfeat[:, 8], dfeat[:, 9] = gs[0], gs[1], gs[2], gs[3], gs[4]
        dfeat[:, 10:13], dfeat[:, 13] = gs[5], gs[6]
        g["mu"] += gs[7]
    L.orc_project_bwd(N, _d(scene.mu)[1], _d(scene.log_s)[1], _d(scene.quat)[1],
                      _d(scene.logit_o)[1], keep[4][1], keep[0][1], keep[1][1],
                      dgeom.ctypes.data_as(_dp), np.ascontiguousarray(dfeat[:, 0]).ctypes.data_as(_dp),
                      g["mu"].ctypes.data_as(_dp), g["log_s"].ctypes.data_as(_dp),
                      g["quat"].ctypes.data_as(_dp), g["logit_o"].ctypes.data_as(_dp))
    g["normal"] += dfeat[:, 1:4]
    g["base"] += dfeat[:, 4:7]
    g["rough"] += dfeat[:, 7]
    g["metal"] += dfeat[:, 8]
    g["sss"] += dfeat[:, 9]
    g["vis"] += dfeat[:, 14]
    dLs, dLin = dfeat[:, 10:13], dfeat[:, 13].copy()
    if dlin_extra is not None:
        dLin += dlin_extra
    if dvis_extra is not None:
        g["vis"] += dvis_extra
    out["dmlp_out"] = np.concatenate([dLs, dLin[:, None]], axis=1)
    if mlp_out is None:
        dWs, dbs, dX = mlp_backward(spec, acts, y, Ls, dLs, dLin, bf16=bf16)
        gi = input_grads(kind, dX, scene.mu, C, pair.light, scene.quat, scene.log_s)
        g["mu"] += gi[0]
        g["normal"] += gi[1]
        g["vis"] += gi[2]
        if kind == "paper":
            g["quat"] += gi[3]
            g["log_s"] += gi[4]
        out["dW"], out["db"] = dWs, dbs
    out["dgeom"], out["dfeat"] = dgeom, dfeat
    out["grads"] = g
    return out


def render_workload_pair(wl, p, **kw):
    pair = wl.pairs[p]
    return render_pair(wl.scenes[pair.scene], pair, wl.mlp, Cfg(tile=wl.tile), **kw)


def brdf(n, wo, wi, base, rough, metal):
    fs = np.zeros(3)
    fd = np.zeros(3)
    lib().orc_brdf(_d(n)[1], _d(wo)[1], _d(wi)[1], _d(base)[1], float(rough), float(metal),
                   fs.ctypes.data_as(_dp), fd.ctypes.data_as(_dp))
    return fs, fd


def shade(gbuf, has, pixels, pair, cfg=DEFAULT_CFG, dimg=None):
    P = gbuf.shape[0]
    img = np.zeros((P, 3))
    dg = np.zeros((P, 16)) if dimg is not None else None
    keep = [_d(gbuf), _i(has), _i(pixels), _d(cam_array(pair)), _d(np.asarray(pair.light, np.float64)),
            _d(cfg.array())]
    lib().orc_shade(P, *[p for _, p in keep], img.ctypes.data_as(_dp),
                    _d(dimg)[1] if dimg is not None else None,
                    dg.ctypes.data_as(_dp) if dg is not None else None)
    return img, dg


def covariance(log_s, quat):
    S = np.zeros(9)
    lib().orc_covariance(_d(log_s)[1], _d(quat)[1], S.ctypes.data_as(_dp))
    return S.reshape(3, 3)


def bin_sort(item_pair, trect, dkey, tiles_x, tile_off, total_tiles, capacity=None):
    """Plain stable sort of (tile, depth key, item) instances; see orc_bin."""
    item_pair, ipp = _i(item_pair)
    trect, trp = _i(trect)
    dkey, dkp = _u(dkey)
    tiles_x, txp = _i(tiles_x)
    tile_off, top = _i(tile_off)
    n_items = item_pair.shape[0]
    r = trect.reshape(-1, 4)
    ok = (r[:, 0] <= r[:, 1]) & (r[:, 2] <= r[:, 3])
    n = int(((r[:, 1] - r[:, 0] + 1) * (r[:, 3] - r[:, 2] + 1) * ok).sum())
    cap = n if capacity is None else capacity
    keys = np.zeros(max(cap, 1), np.uint32)
    vals = np.zeros(max(cap, 1), np.uint32)
    ranges = np.zeros(2 * total_tiles, np.uint32)
    got = lib().orc_bin(n_items, ipp, trp, dkp, txp, top, int(total_tiles), int(cap),
                        keys.ctypes.data_as(_up), vals.ctypes.data_as(_up),
                        ranges.ctypes.data_as(_up))
    return int(got), keys[:min(cap, n)], vals[:min(cap, n)], ranges.reshape(-1, 2)
