"""Seeded synthetic inputs for the SSS Gaussian-splatting OLAT render.

This module draws scenes, cameras, point lights, MLP weights and upstream
gradients. It holds none of the method's arithmetic (no projection,
compositing, shading or network evaluation): both the CUDA path and the FP64
oracle consume what it returns, and neither imports the other.

Every floating-point array is rounded to a float32-representable value and
returned as float64, so the two sides start from bit-identical inputs (the GPU
casts to float32 exactly, the oracle keeps float64).

Workload shapes follow the paper's synthetic OLAT set (800x800 images, cameras
at a fixed distance, point lights on a sphere; Section 4.1 "Dataset") and the
five configurations this library is measured on:

  c1  1,024 Gaussians in a shell r in [0.8, 1.0], 128x128, MLP 9-32-32-4 FP32
  c2  100K Gaussians on a seeded SH blob, 512x512, MLP 9-64-64-64-4 FP32
  c3  300K Gaussians on the blob, 800x800, MLP PE6(50->64)-128x4-4 BF16
  c4  the c3 scene with 64 Fibonacci view/light pairs at 800x800
  c5  8 blob scenes (50K..1M Gaussians) x 8 pairs at {400..1600}^2
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Scene", "Pair", "MLPSpec", "Workload", "make_workload", "look_at",
    "pinhole", "fibonacci_sphere", "random_dimg", "synthetic_bin_inputs",
    "f32", "FEATURE_NAMES",
]

# G-buffer feature order shared by the documentation of both sides.
FEATURE_NAMES = ("depth", "n0", "n1", "n2", "b0", "b1", "b2", "rough",
                 "metal", "sss", "Ls0", "Ls1", "Ls2", "Lin", "vis")


def f32(a) -> np.ndarray:
    """Round to float32 and return float64 holding exactly that value."""
    return np.asarray(a, dtype=np.float64).astype(np.float32).astype(np.float64)


@dataclass
class Scene:
    """Per-Gaussian parameters (float64 arrays holding float32 values)."""
    mu: np.ndarray        # N x 3 mean
    log_s: np.ndarray     # N x 3 log scale
    quat: np.ndarray      # N x 4 (w, x, y, z), not necessarily unit
    logit_o: np.ndarray   # N opacity logit
    normal: np.ndarray    # N x 3
    base: np.ndarray      # N x 3 base colour
    rough: np.ndarray     # N
    metal: np.ndarray     # N
    sss: np.ndarray       # N subsurfaceness
    vis: np.ndarray       # N visibility scalar

    @property
    def N(self) -> int:
        return int(self.mu.shape[0])

    def arrays(self):
        return dict(mu=self.mu, log_s=self.log_s, quat=self.quat,
                    logit_o=self.logit_o, normal=self.normal, base=self.base,
                    rough=self.rough, metal=self.metal, sss=self.sss,
                    vis=self.vis)

    def subset(self, idx) -> "Scene":
        return Scene(**{k: v[idx].copy() for k, v in self.arrays().items()})


@dataclass
class Pair:
    """One OLAT view/light pair: pinhole camera (world->camera) + point light."""
    R: np.ndarray         # 3 x 3 world->camera rotation (rows: right, down, forward)
    t: np.ndarray         # 3 translation, x_cam = R x_world + t
    fx: float
    fy: float
    cx: float
    cy: float
    W: int
    H: int
    light: np.ndarray     # 3 light position
    scene: int = 0        # index of the scene the pair renders

    @property
    def center(self) -> np.ndarray:
        return -self.R.T @ self.t


@dataclass
class MLPSpec:
    """Residual / incident-light MLP: layer weights W[l] (out x in) and b[l]."""
    kind: str                 # "basic" (9 inputs), "pe6" (50 padded to 64) or "paper" (42 padded to 48)
    n_in: int                 # input width seen by the first layer
    widths: list              # hidden widths
    weights: list = field(default_factory=list)
    biases: list = field(default_factory=list)
    precision: str = "fp32"   # "fp32" or "bf16"


@dataclass
class Workload:
    name: str
    scenes: list
    pairs: list
    mlp: MLPSpec
    tile: int = 16
    target_scene: Scene | None = None   # perturbed scene for the L1 target
    n_lights: int = 1        # lights per view: pairs come in runs of n_lights sharing one camera


# --------------------------------------------------------------------------
# camera helpers (geometry of the synthetic light stage, not of the method)
# --------------------------------------------------------------------------

def look_at(center, target=(0.0, 0.0, 0.0), up=(0.0, 0.0, 1.0)):
    """OpenCV-style world->camera (x right, y down, z forward)."""
    c = np.asarray(center, np.float64)
    f = np.asarray(target, np.float64) - c
    f /= np.linalg.norm(f)
    up = np.asarray(up, np.float64)
    r = np.cross(f, up)
    if np.linalg.norm(r) < 1e-9:          # looking straight up/down
        r = np.cross(f, np.array([0.0, 1.0, 0.0]))
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f])
    R = f32(R)
    t = f32(-R @ c)
    return R, t


def pinhole(W: int, H: int, fov_y_deg: float = 50.0):
    fy = (H / 2.0) / math.tan(math.radians(fov_y_deg) / 2.0)
    return float(f32(fy)), float(f32(fy)), W / 2.0, H / 2.0


def fibonacci_sphere(n: int, radius: float, upper: bool = False) -> np.ndarray:
    """n points of a Fibonacci lattice on a sphere (or its z>0 half)."""
    i = np.arange(n, dtype=np.float64) + 0.5
    if upper:
        z = 1.0 - i / n          # z in (0, 1)
    else:
        z = 1.0 - 2.0 * i / n
    rho = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = i * math.pi * (3.0 - math.sqrt(5.0))
    return radius * np.stack([rho * np.cos(phi), rho * np.sin(phi), z], axis=1)


def _make_pair(cam_pos, light_pos, W, H, scene=0) -> Pair:
    R, t = look_at(cam_pos)
    fx, fy, cx, cy = pinhole(W, H)
    return Pair(R=R, t=t, fx=fx, fy=fy, cx=cx, cy=cy, W=W, H=H,
                light=f32(light_pos), scene=scene)


# --------------------------------------------------------------------------
# scene geometry
# --------------------------------------------------------------------------

def _unit(rng, n):
    v = rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _real_sh(l, m, theta, phi):
    """Unnormalised real spherical harmonic (shape only; rescaled later)."""
    from scipy.special import lpmv
    p = lpmv(abs(m), l, np.cos(theta))
    if m > 0:
        return p * np.cos(m * phi)
    if m < 0:
        return p * np.sin(-m * phi)
    return p


class _Blob:
    """r(w) = 1 + amp * sum_k Y_k(w) / max|Y_k| with seeded degree/order."""

    def __init__(self, rng, n_bumps=4, amp=0.1):
        self.terms = []
        th = np.linspace(0.0, math.pi, 361)
        ph = np.linspace(0.0, 2 * math.pi, 721)
        TH, PH = np.meshgrid(th, ph, indexing="ij")
        for _ in range(n_bumps):
            l = int(rng.integers(2, 6))
            m = int(rng.integers(-l, l + 1))
            mx = np.abs(_real_sh(l, m, TH, PH)).max()
            self.terms.append((l, m, amp / mx))

    def radius(self, d):
        theta = np.arccos(np.clip(d[:, 2], -1.0, 1.0))
        phi = np.arctan2(d[:, 1], d[:, 0])
        r = np.ones(d.shape[0])
        for l, m, s in self.terms:
            r = r + s * _real_sh(l, m, theta, phi)
        return r

    def implicit(self, x):
        nrm = np.linalg.norm(x, axis=1)
        return nrm - self.radius(x / nrm[:, None])

    def normals(self, x, h=1e-6):
        g = np.zeros_like(x)
        for k in range(3):
            e = np.zeros(3)
            e[k] = h
            g[:, k] = (self.implicit(x + e) - self.implicit(x - e)) / (2 * h)
        return g / np.linalg.norm(g, axis=1, keepdims=True)


def _materials(rng, N, metal_zero):
    base = rng.uniform(0.0, 1.0, (N, 3))
    rough = rng.uniform(0.1, 1.0, N)
    metal = np.zeros(N) if metal_zero else rng.uniform(0.0, 1.0, N)
    sss = rng.uniform(0.0, 1.0, N)
    return base, rough, metal, sss


def shell_scene(seed: int, N: int = 1024) -> Scene:
    rng = np.random.Generator(np.random.PCG64(seed))
    d = _unit(rng, N)
    r = (rng.uniform(0.8 ** 3, 1.0, N)) ** (1.0 / 3.0)
    mu = d * r[:, None]
    log_s = rng.normal(-3.5, 0.3, (N, 3))
    q = rng.standard_normal((N, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    logit_o = rng.normal(0.0, 1.0, N)
    base, rough, metal, sss = _materials(rng, N, metal_zero=True)
    return Scene(mu=f32(mu), log_s=f32(log_s), quat=f32(q), logit_o=f32(logit_o),
                 normal=f32(d), base=f32(base), rough=f32(rough), metal=f32(metal),
                 sss=f32(sss), vis=f32(np.ones(N)))


def blob_scene(seed: int, N: int, scale_ref: float = 1e5) -> Scene:
    """Gaussians on a seeded SH blob; log-scale mean shifted by -0.5 ln(N/1e5)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    blob = _Blob(rng)
    d = _unit(rng, N)
    x = d * blob.radius(d)[:, None]
    n = blob.normals(x)
    shift = -0.5 * math.log(N / scale_ref)
    log_s = rng.normal(-3.5 + shift, 0.3, (N, 3))
    q = rng.standard_normal((N, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    logit_o = rng.normal(0.0, 1.0, N)
    base, rough, metal, sss = _materials(rng, N, metal_zero=False)
    vis = rng.uniform(0.0, 1.0, N)
    return Scene(mu=f32(x), log_s=f32(log_s), quat=f32(q), logit_o=f32(logit_o),
                 normal=f32(n), base=f32(base), rough=f32(rough), metal=f32(metal),
                 sss=f32(sss), vis=f32(vis))


def perturbed(scene: Scene, seed: int) -> Scene:
    """Target scene: mu + N(0,0.01), log_s + N(0,0.05), base + N(0,0.05)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    s = scene.subset(slice(None))
    s.mu = f32(s.mu + rng.normal(0, 0.01, s.mu.shape))
    s.log_s = f32(s.log_s + rng.normal(0, 0.05, s.log_s.shape))
    s.base = f32(np.clip(s.base + rng.normal(0, 0.05, s.base.shape), 0.0, 1.0))
    return s


def mlp_spec(seed: int, kind: str, widths, precision="fp32", std=None) -> MLPSpec:
    """Weights ~ N(0, std) (0.1 by default, He-scaled for 128-wide layers);
    biases 0 except the incident-light output, biased +0.5 so most Gaussians
    receive light at initialisation.

    kind "paper" (widths ignored): the six matrices of the paper's network in
    the order W0 64x48, W1 32x64, W2 32x32 (trunk), W3 32x32 (incident
    hidden), W4 1x32 (incident output), W5 3x32 (SSS output), He-scaled."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if kind == "paper":
        shapes = [(64, 48), (32, 64), (32, 32), (32, 32), (1, 32), (3, 32)]
        fan_in = [42, 64, 32, 32, 32, 32]
        Ws, bs = [], []
        for (o, i), fi in zip(shapes, fan_in):
            W = rng.normal(0.0, std if std is not None else math.sqrt(2.0 / fi), (o, i))
            if i == 48:
                W[:, 42:] = 0.0      # padded inputs carry no weight
            Ws.append(f32(W))
            bs.append(f32(np.zeros(o)))
        bs[4] = f32(np.full(1, 0.5))
        return MLPSpec(kind=kind, n_in=48, widths=[64, 32, 32], weights=Ws, biases=bs, precision=precision)
    n_in = 9 if kind == "basic" else 64
    dims = [n_in] + list(widths) + [4]
    Ws, bs = [], []
    for l in range(len(dims) - 1):
        sd = std if std is not None else (0.1 if kind == "basic"
                                          else math.sqrt(2.0 / (50 if l == 0 else dims[l])))
        W = rng.normal(0.0, sd, (dims[l + 1], dims[l]))
        if kind == "pe6" and l == 0:
            W[:, 50:] = 0.0      # padded inputs carry no weight
        b = np.zeros(dims[l + 1])
        if l == len(dims) - 2:
            b[3] = 0.5
        Ws.append(f32(W))
        bs.append(f32(b))
    return MLPSpec(kind=kind, n_in=n_in, widths=list(widths), weights=Ws,
                   biases=bs, precision=precision)


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

def _hemisphere_dir(rng, zmin=0.15):
    while True:
        v = _unit(rng, 1)[0]
        if v[2] > zmin:
            return v


def light_stage(radius: float = 4.0, rings: int = 7, per_ring: int = 16) -> np.ndarray:
    """The synthetic light stage of Sec. 4.1: `rings` rings of `per_ring` point
    lights on the upper hemisphere (elevations evenly spaced strictly between
    the horizon and the pole, rings offset by half a step in azimuth)."""
    out = []
    for r in range(rings):
        el = (r + 0.5) * (0.5 * math.pi) / rings
        for k in range(per_ring):
            az = 2.0 * math.pi * (k + 0.5 * (r % 2)) / per_ring
            out.append(radius * np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)]))
    return np.array(out)


def make_workload(name: str, *, N: int | None = None, res=None,
                  n_pairs: int | None = None, seed_offset: int = 0, net: str | None = None,
                  n_views: int | None = None, n_lights: int | None = None) -> Workload:
    """Build configuration `name` ("c1".."c6"); N/res/n_pairs shrink it for tests.
    For c5, `res` may be a tuple of resolutions to draw from. net="paper"
    replaces the configuration's network by the paper's (App. E). c6 is a
    light-stage batch of n_views views (default 8) under n_lights lights each
    (default 8) of the 112-light stage."""
    wl = _make_workload(name, N=N, res=res, n_pairs=n_pairs, seed_offset=seed_offset, n_views=n_views,
                        n_lights=n_lights)
    if net == "paper":   # keeps the configuration's precision (BF16 tensor cores for c3-c5)
        wl.mlp = mlp_spec(int(name[1]) * 1000 + seed_offset + 13, "paper", [], precision=wl.mlp.precision)
    elif net is not None:
        raise ValueError(f"unknown network {net!r}")
    return wl


def _make_workload(name: str, *, N: int | None = None, res=None,
                   n_pairs: int | None = None, seed_offset: int = 0, n_views: int | None = None,
                   n_lights: int | None = None) -> Workload:
    idx = int(name[1])
    seed = idx * 1000 + seed_offset
    rng = np.random.Generator(np.random.PCG64(seed + 7))
    if name == "c1":
        n = N or 1024
        W = res or 128
        scene = shell_scene(seed, n)
        cam = 3.0 * np.array([1.0, 0.0, 1.0]) / math.sqrt(2.0)
        light = 4.0 * np.array([1.0, 0.5, 1.0]) / 1.5
        pairs = [_make_pair(cam, light, W, W)]
        mlp = mlp_spec(seed + 11, "basic", [32, 32])
        return Workload(name, [scene], pairs, mlp, 16, perturbed(scene, seed + 1))
    if name == "c2":
        n = N or 100_000
        W = res or 512
        scene = blob_scene(seed, n)
        cam = 3.0 * _hemisphere_dir(rng)
        light = 4.0 * _unit(rng, 1)[0]
        pairs = [_make_pair(cam, light, W, W)]
        mlp = mlp_spec(seed + 11, "basic", [64, 64, 64])
        return Workload(name, [scene], pairs, mlp, 16, perturbed(scene, seed + 1))
    if name == "c3":
        n = N or 300_000
        W = res or 800
        scene = blob_scene(seed, n)
        cam = 3.0 * _hemisphere_dir(rng)
        light = 4.0 * _unit(rng, 1)[0]
        pairs = [_make_pair(cam, light, W, W)]
        mlp = mlp_spec(seed + 11, "pe6", [128, 128, 128, 128], precision="bf16")
        return Workload(name, [scene], pairs, mlp, 16, None)
    if name == "c4":
        n = N or 300_000
        W = res or 800
        P = n_pairs or 64
        scene = blob_scene(3000 + seed_offset, n)      # the c3 scene
        cams = fibonacci_sphere(P, 3.0, upper=True)
        lights = fibonacci_sphere(P, 4.0, upper=False)
        perm = rng.permutation(P)
        pairs = [_make_pair(cams[i], lights[perm[i]], W, W) for i in range(P)]
        mlp = mlp_spec(3000 + seed_offset + 11, "pe6", [128, 128, 128, 128],
                       precision="bf16")
        return Workload(name, [scene], pairs, mlp, 16, None)
    if name == "c5":
        counts = [50_000, 100_000, 200_000, 300_000, 500_000, 700_000, 850_000, 1_000_000]
        if N is not None:
            counts = [max(64, int(c * N / 1_000_000)) for c in counts]
        per = n_pairs or 8
        scenes, pairs = [], []
        for s, c in enumerate(counts):
            scenes.append(blob_scene(seed + 100 * s, c))
            cams = fibonacci_sphere(per, 3.0, upper=True)
            lights = fibonacci_sphere(per, 4.0)
            choices = list(res) if isinstance(res, (tuple, list)) else ([res] if res else [400, 800, 1200, 1600])
            for k in range(per):
                r = int(rng.choice(choices))
                rc = (k + s) % per
                pairs.append(_make_pair(cams[k], lights[rc], r, r, scene=s))
        mlp = mlp_spec(seed + 11, "pe6", [128, 128, 128, 128], precision="bf16")
        return Workload(name, scenes, pairs, mlp, 16, None)
    if name == "c6":
        n = N or 300_000
        W = res or 800
        V = n_views or 8
        L = n_lights or 8
        scene = blob_scene(3000 + seed_offset, n)      # the c3 scene
        cams = fibonacci_sphere(V, 3.0, upper=True)
        stage = light_stage(4.0)
        pairs = []
        for v in range(V):
            for li in rng.choice(len(stage), size=L, replace=False):
                pairs.append(_make_pair(cams[v], stage[li], W, W))
        mlp = mlp_spec(3000 + seed_offset + 11, "pe6", [128, 128, 128, 128], precision="bf16")
        return Workload(name, [scene], pairs, mlp, 16, None, n_lights=L)
    raise ValueError(f"unknown workload {name!r}")


def vis_sh_coeffs(seed: int, N: int) -> np.ndarray:
    """Seeded coefficients of a degree-3 SH visibility term per Gaussian
    (N x 16): a constant band giving v in [0.3, 0.9] plus small higher bands."""
    rng = np.random.Generator(np.random.PCG64(seed))
    c = rng.normal(0.0, 0.08, (N, 16))
    c[:, 0] = rng.uniform(0.3, 0.9, N) * 2.0 * math.sqrt(math.pi)   # the constant band's basis value is 1 / (2 sqrt(pi))
    return f32(c)


def random_dimg(seed: int, n_pixels: int) -> np.ndarray:
    """Seeded upstream image gradient dL/d(image), float32 values, P x 3."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return f32(rng.uniform(-1.0, 1.0, (n_pixels, 3)))


def synthetic_bin_inputs(seed: int, n_pairs: int, N: int, tiles_x: int, tiles_y: int,
                         tie_fraction: float = 0.2, cull_fraction: float = 0.1):
    """Per-(pair, Gaussian) tile rectangles and float32 depth keys for the
    bin/sort stage, drawn directly (no projection): footprint sizes follow the
    300K-blob workload (1-6 tiles a side), depths cluster so that many keys tie
    exactly, and a fraction of entries is culled (empty rectangle).

    Returns rect (n_pairs*N x 4 int32: tx0, tx1, ty0, ty1, inclusive, tx0>tx1
    means culled) and depth (n_pairs*N float32)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    M = n_pairs * N
    w = rng.integers(1, 7, M)
    h = rng.integers(1, 7, M)
    tx0 = rng.integers(0, tiles_x, M)
    ty0 = rng.integers(0, tiles_y, M)
    tx1 = np.minimum(tx0 + w - 1, tiles_x - 1)
    ty1 = np.minimum(ty0 + h - 1, tiles_y - 1)
    cull = rng.uniform(size=M) < cull_fraction
    tx0 = np.where(cull, 1, tx0)
    tx1 = np.where(cull, 0, tx1)
    depth = rng.uniform(1.5, 4.5, M).astype(np.float32)
    ties = rng.uniform(size=M) < tie_fraction
    pool = rng.uniform(1.5, 4.5, 16).astype(np.float32)
    depth[ties] = pool[rng.integers(0, 16, int(ties.sum()))]
    rect = np.stack([tx0, tx1, ty0, ty1], axis=1).astype(np.int32)
    return rect, depth
