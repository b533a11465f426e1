"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these re-types the oracle's own formula: each checks a closed form,
an invariant, a brute-force/library result or a quadrature that a dropped
term, wrong sign, wrong index or transposed operand would break.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
import scenegen as sg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _pair_looking_down_z(W=64, H=64, fx=80.0, light=(0.0, 0.0, -5.0)):
    """Camera at the origin looking along +z (R = I, t = 0)."""
    return sg.Pair(R=np.eye(3), t=np.zeros(3), fx=fx, fy=fx, cx=W / 2, cy=H / 2, W=W, H=H,
                   light=np.asarray(light, float))


def _scene(mu, log_s, quat, logit, **kw):
    N = len(mu)
    d = dict(mu=np.asarray(mu, float).reshape(N, 3), log_s=np.asarray(log_s, float).reshape(N, 3),
             quat=np.asarray(quat, float).reshape(N, 4), logit_o=np.asarray(logit, float).reshape(N),
             normal=np.tile([0.0, 0.0, -1.0], (N, 1)), base=np.full((N, 3), 0.5),
             rough=np.full(N, 0.5), metal=np.zeros(N), sss=np.full(N, 0.5), vis=np.ones(N))
    d.update({k: np.asarray(v, float) for k, v in kw.items()})
    return sg.Scene(**d)


# ---------------------------------------------------------------- covariance

def test_identity_quaternion_gives_diagonal_covariance():
    s = np.array([-1.0, -2.0, -0.5])
    S = O.covariance(s, [1.0, 0, 0, 0])
    assert np.allclose(S, np.diag(np.exp(2 * s)), atol=1e-15)


def test_quarter_turn_about_z_swaps_x_and_y_scales():
    s = np.array([-1.0, -2.0, -0.5])
    q = [math.cos(math.pi / 4), 0, 0, math.sin(math.pi / 4)]
    S = O.covariance(s, q)
    e = np.exp(2 * s)
    assert np.allclose(S, np.diag([e[1], e[0], e[2]]), atol=1e-15)


def test_covariance_is_rotation_conjugate_and_unnormalised_quaternion_ok():
    rng = np.random.default_rng(3)
    for _ in range(20):
        q = rng.standard_normal(4) * 3.7     # not unit: the oracle normalises
        s = rng.normal(-2, 0.5, 3)
        S = O.covariance(s, q)
        # isotropic scales: any rotation gives s^2 I (R R^T = I)
        Si = O.covariance(np.full(3, s[0]), q)
        assert np.allclose(Si, np.exp(2 * s[0]) * np.eye(3), atol=1e-14)
        # eigenvalues are the squared scales
        assert np.allclose(np.sort(np.linalg.eigvalsh(S)), np.sort(np.exp(2 * s)), rtol=1e-12)
        # compare with scipy's quaternion rotation (library routine; scalar-last)
        from scipy.spatial.transform import Rotation
        R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        assert np.allclose(S, R @ np.diag(np.exp(2 * s)) @ R.T, atol=1e-14)


# ---------------------------------------------------------------- EWA (Eq. 2)

def test_isotropic_gaussian_on_axis_closed_form():
    z, s, f, dil = 4.0, 0.05, 100.0, 0.3
    pair = _pair_looking_down_z(fx=f)
    sc = _scene([[0, 0, z]], [[math.log(s)] * 3], [[1, 0, 0, 0]], [2.0])
    cfg = O.Cfg(dilation=dil)
    proj, rect, _ = O.project(sc, pair, cfg)
    var = (f * s / z) ** 2 + dil
    assert proj[0, 0] == pytest.approx(pair.cx) and proj[0, 1] == pytest.approx(pair.cy)
    assert proj[0, 13] == pytest.approx(var, rel=1e-14)
    assert proj[0, 14] == pytest.approx(0.0, abs=1e-15)
    assert proj[0, 2] == pytest.approx(1 / var, rel=1e-13)
    assert proj[0, 4] == pytest.approx(1 / var, rel=1e-13)
    assert proj[0, 6] == pytest.approx(z)
    o = 1 / (1 + math.exp(-2.0))
    assert proj[0, 5] == pytest.approx(o)
    assert proj[0, 7] == pytest.approx(math.log(255 * o), rel=1e-6)  # alpha_min is f32(1/255)


@pytest.mark.parametrize("mu,scales", [([0.4, 0.2, -0.1], [0.004, 0.002, 0.006]),
                                       ([0.4, 0.9, 0.6], [0.004, 0.002, 0.02])])
def test_off_axis_projection_matches_monte_carlo(mu, scales):
    """Small Gaussian off axis: EWA covariance ~ covariance of projected samples.
    The second case lies far off axis in both image directions (|t_x / t_z|,
    |t_y / t_z| ~ 0.15, 0.27) and is elongated, so every entry of the
    projection Jacobian's depth column shapes the footprint."""
    rng = np.random.default_rng(11)
    pair = sg._make_pair([0.3, -2.5, 1.2], [0, 0, 4], 256, 256)
    mu = np.array([mu])
    ls = np.log([scales])
    q = np.array([[0.8, 0.3, -0.4, 0.2]])
    sc = _scene(mu, ls, q, [1.0])
    proj, _, _ = O.project(sc, pair, O.Cfg(dilation=0.0))
    S = O.covariance(ls[0], q[0])
    X = rng.multivariate_normal(mu[0], S, size=400_000)
    t = X @ pair.R.T + pair.t
    uv = np.stack([pair.fx * t[:, 0] / t[:, 2] + pair.cx, pair.fy * t[:, 1] / t[:, 2] + pair.cy], 1)
    C = np.cov(uv.T)
    E = np.array([[proj[0, 13], proj[0, 14]], [proj[0, 14], proj[0, 15]]])
    assert np.allclose(E, C, rtol=0.02, atol=0.02 * np.abs(C).max())
    assert np.allclose(uv.mean(0), proj[0, :2], atol=0.02)


def test_near_plane_and_opacity_culling():
    pair = _pair_looking_down_z()
    sc = _scene([[0, 0, 0.1], [0, 0, 3.0], [0, 0, 3.0]], [[-2] * 3] * 3,
                [[1, 0, 0, 0]] * 3, [2.0, -8.0, 2.0])
    _, rect, _ = O.project(sc, pair)
    valid = rect[:, 0] <= rect[:, 1]
    assert list(valid) == [False, False, True]    # behind z_near; o < 1/255; ok


# ---------------------------------------------------------------- alpha (Eq. 3)

def test_lone_gaussian_peak_alpha_equals_opacity():
    """Mean on a pixel centre, no dilation: alpha = o there (Eq. 3 with one term)."""
    pair = _pair_looking_down_z(W=32, H=32, fx=80.0)
    # pixel (16, 16) centre = (16.5, 16.5): put the mean there
    z = 3.0
    x = (16.5 - pair.cx) * z / pair.fx
    sc = _scene([[x, x, z]], [[-2.5] * 3], [[1, 0, 0, 0]], [0.3], sss=[1.0])
    r = O.render_pair(sc, pair, sg.mlp_spec(1, "basic", [8]), O.Cfg(dilation=0.0),
                      pixels=np.array([[16, 16]], np.int32), mlp_out=np.array([[0.2, 0.4, 0.6, 1.0]]))
    o = 1 / (1 + math.exp(-0.3))
    T = r["gbuf"][0, 15]
    assert 1 - T == pytest.approx(o, rel=1e-14)
    # every composited channel is o * feature
    assert r["gbuf"][0, 9] == pytest.approx(o * 1.0, rel=1e-14)      # sss
    assert r["gbuf"][0, 0] == pytest.approx(o * z, rel=1e-14)        # depth
    # shading with sss = 1 reduces Eq. 7 to L_out = L_SSS; image = A * L_SSS
    assert np.allclose(r["img"][0], o * np.array([0.2, 0.4, 0.6]), rtol=1e-13)


def test_isotropic_alpha_falloff_closed_form():
    """Isotropic Gaussian on the optical axis: Sigma' = ((f s / z)^2 + dil) I,
    so alpha at a pixel centre a distance r from the mean is
    o exp(-r^2 / (2 var)) (Eq. 3's alpha with the EWA footprint of Eq. 2)."""
    z, s, f, dil = 3.0, 0.06, 60.0, 0.3
    pair = _pair_looking_down_z(W=32, H=32, fx=f)
    sc = _scene([[0, 0, z]], [[math.log(s)] * 3], [[1, 0, 0, 0]], [0.0], sss=[1.0])
    pix = np.array([[i, j] for i in range(12, 21) for j in range(12, 21)], np.int32)
    r = O.render_pair(sc, pair, sg.mlp_spec(1, "basic", [8]), O.Cfg(dilation=dil), pixels=pix,
                      mlp_out=np.zeros((1, 4)))
    var = (f * s / z) ** 2 + dil
    r2 = (pix[:, 0] + 0.5 - pair.cx) ** 2 + (pix[:, 1] + 0.5 - pair.cy) ** 2
    expect = 0.5 * np.exp(-r2 / (2 * var))
    seen = expect >= np.float32(1 / 255) * (1 + 1e-6)
    assert seen.sum() >= 20
    assert np.allclose(1 - r["gbuf"][seen, 15], expect[seen], rtol=1e-12)


def test_anisotropic_alpha_follows_the_projected_covariance():
    """Rotated, anisotropic, off-axis Gaussian on a non-square image: alpha at
    every pixel equals o exp(-d^T Sigma'^-1 d / 2), with Sigma' the projected
    covariance (pinned against Monte Carlo above), its inverse taken by
    numpy, and d the offset from the pinhole projection of the mean."""
    W, H, f = 48, 40, 60.0
    pair = sg.Pair(R=np.eye(3), t=np.zeros(3), fx=f, fy=f, cx=W / 2, cy=H / 2, W=W, H=H,
                   light=np.array([0.0, 0.0, -5.0]))
    mu = np.array([0.3, -0.2, 3.0])
    sc = _scene([mu], [[-2.6, -3.4, -3.0]], [[0.8, 0.3, -0.4, 0.2]], [0.0], sss=[1.0])
    proj, _, _ = O.project(sc, pair)
    E = np.array([[proj[0, 13], proj[0, 14]], [proj[0, 14], proj[0, 15]]])
    assert abs(E[0, 1]) > 0.1 * math.sqrt(E[0, 0] * E[1, 1])    # the footprint is tilted
    m = np.array([f * mu[0] / mu[2] + pair.cx, f * mu[1] / mu[2] + pair.cy])
    pix = O.all_pixels(W, H)
    r = O.render_pair(sc, pair, sg.mlp_spec(1, "basic", [8]), pixels=pix, mlp_out=np.zeros((1, 4)))
    d = m[None, :] - (pix + 0.5)
    q = np.einsum("ni,ij,nj->n", d, np.linalg.inv(E), d)
    expect = 0.5 * np.exp(-0.5 * q)
    seen = expect >= np.float32(1 / 255) * (1 + 1e-6)
    assert seen.sum() >= 30
    assert np.allclose(1 - r["gbuf"][seen, 15], expect[seen], rtol=1e-11)
    assert np.all(r["gbuf"][expect < np.float32(1 / 255) * (1 - 1e-6), 15] == 1.0)


def test_opaque_gaussian_alpha_clamps_at_alpha_max():
    """Mean on a pixel centre, opacity above alpha_max: alpha = 0.99 there."""
    pair = _pair_looking_down_z(W=32, H=32, fx=80.0)
    z = 3.0
    x = (16.5 - pair.cx) * z / pair.fx
    sc = _scene([[x, x, z]], [[-2.5] * 3], [[1, 0, 0, 0]], [8.0])
    r = O.render_pair(sc, pair, sg.mlp_spec(1, "basic", [8]), O.Cfg(dilation=0.0),
                      pixels=np.array([[16, 16]], np.int32), mlp_out=np.zeros((1, 4)))
    assert 1 - r["gbuf"][0, 15] == pytest.approx(float(np.float32(0.99)), rel=1e-14)   # alpha_max is f32(0.99)


# ---------------------------------------------------------------- compositing (Eq. 3)

def test_weights_telescope_to_one_minus_T_everywhere():
    wl = sg.make_workload("c1")
    sc = wl.scenes[0].subset(slice(None))
    sc.sss = np.ones(sc.N)      # the sss channel then accumulates sum_i w_i
    r = O.render_pair(sc, wl.pairs[0], wl.mlp)
    T = r["gbuf"][:, 15]
    assert np.abs(r["gbuf"][:, 9] - (1 - T)).max() < 1e-12
    assert (r["ncontrib"] > 0).mean() > 0.3


def test_two_coincident_gaussians_closed_form():
    pair = _pair_looking_down_z(W=16, H=16, fx=40.0)
    z1, z2 = 2.0, 2.5
    # both centred on the ray through pixel (8, 8)
    x1 = (8.5 - pair.cx) / pair.fx
    sc = _scene([[x1 * z1, x1 * z1, z1], [x1 * z2, x1 * z2, z2]], [[-1.5] * 3] * 2,
                [[1, 0, 0, 0]] * 2, [0.5, 1.5], base=[[0.9, 0.1, 0.2], [0.1, 0.8, 0.3]])
    r = O.render_pair(sc, pair, sg.mlp_spec(1, "basic", [8]), O.Cfg(dilation=0.0),
                      pixels=np.array([[8, 8]], np.int32), mlp_out=np.zeros((2, 4)))
    a1 = 1 / (1 + math.exp(-0.5))
    a2 = 1 / (1 + math.exp(-1.5))
    c1, c2 = np.array([0.9, 0.1, 0.2]), np.array([0.1, 0.8, 0.3])
    expect = a1 * c1 + (1 - a1) * a2 * c2
    assert np.allclose(r["gbuf"][0, 4:7], expect, rtol=1e-13)
    assert r["gbuf"][0, 15] == pytest.approx((1 - a1) * (1 - a2), rel=1e-13)


def test_equal_depth_ties_composite_in_storage_order():
    """Two Gaussians at the same mean (equal float32 depth keys) composite in
    storage order: C = a0 c0 + (1 - a0) a1 c1 with Gaussian 0 in front (the
    stable sort's tie rule); a0 != a1 makes the other order differ."""
    pair = _pair_looking_down_z(W=16, H=16, fx=40.0)
    z = 2.0
    x = (8.5 - pair.cx) / pair.fx * z
    c0, c1 = np.array([0.9, 0.1, 0.2]), np.array([0.1, 0.8, 0.3])
    sc = _scene([[x, x, z]] * 2, [[-1.5] * 3] * 2, [[1, 0, 0, 0]] * 2, [0.5, 1.5], base=[c0, c1])
    r = O.render_pair(sc, pair, sg.mlp_spec(1, "basic", [8]), O.Cfg(dilation=0.0),
                      pixels=np.array([[8, 8]], np.int32), mlp_out=np.zeros((2, 4)))
    assert r["dkey"][0] == r["dkey"][1]
    a0, a1 = 1 / (1 + math.exp(-0.5)), 1 / (1 + math.exp(-1.5))
    assert np.allclose(r["gbuf"][0, 4:7], a0 * c0 + (1 - a0) * a1 * c1, rtol=1e-13)
    assert not np.allclose(a0 * c0 + (1 - a0) * a1 * c1, a1 * c1 + (1 - a1) * a0 * c0, rtol=1e-3)


def test_brute_force_equals_tiled_bitwise_and_tile_size_independent():
    wl = sg.make_workload("c2", N=6000, res=96)
    base = O.render_workload_pair(wl, 0, mode=0)
    for tile in (8, 16, 32):
        r = O.render_pair(wl.scenes[0], wl.pairs[0], wl.mlp, O.Cfg(tile=tile), mode=1)
        assert np.array_equal(r["gbuf"], base["gbuf"])
        assert np.array_equal(r["img"], base["img"])
    assert (base["ncontrib"] > 0).mean() > 0.2


def test_storage_order_permutation_invariance():
    """Storage order only breaks ties of equal float32 depth keys. A random
    permutation that keeps the relative order inside each tie group leaves
    every pixel bit-identical."""
    wl = sg.make_workload("c1")
    sc = wl.scenes[0]
    r0 = O.render_pair(sc, wl.pairs[0], wl.mlp)
    perm = np.random.default_rng(5).permutation(sc.N)       # new slot k holds old perm[k]
    pos = np.empty(sc.N, np.int64)
    pos[perm] = np.arange(sc.N)
    for key in np.unique(r0["dkey"]):
        grp = np.flatnonzero(r0["dkey"] == key)             # old indices, ascending
        if len(grp) > 1:
            slots = np.sort(pos[grp])
            perm[slots] = grp
    assert len(np.unique(r0["dkey"])) < sc.N                # c1 does contain a tie
    r1 = O.render_pair(sc.subset(perm), wl.pairs[0], wl.mlp)
    assert np.array_equal(r0["img"], r1["img"])
    assert np.array_equal(r0["gbuf"], r1["gbuf"])


def test_depth_order_and_stop_rule():
    """Front-to-back order by depth, and the T < T_min stop (before the Gaussian)."""
    pair = _pair_looking_down_z(W=8, H=8, fx=20.0)
    # 12 opaque-ish identical Gaussians on the centre ray, shuffled storage order
    zs = np.array([2.0 + 0.1 * k for k in range(12)])
    perm = np.random.default_rng(2).permutation(12)
    zs = zs[perm]
    x = (4.5 - pair.cx) / pair.fx
    sc = _scene([[x * z, x * z, z] for z in zs], [[-1.0] * 3] * 12, [[1, 0, 0, 0]] * 12,
                [4.0] * 12, rough=zs)   # rough channel carries the depth rank
    r = O.render_pair(sc, pair, sg.mlp_spec(1, "basic", [8]), O.Cfg(dilation=0.0),
                      pixels=np.array([[4, 4]], np.int32), mlp_out=np.zeros((12, 4)))
    a = min(0.99, 1 / (1 + math.exp(-4.0)))
    T, acc, n = 1.0, 0.0, 0
    for z in sorted(zs):
        if T * (1 - a) < np.float32(1e-4):
            break
        acc += T * a * z
        T *= 1 - a
        n += 1
    assert r["ncontrib"][0] == n and 0 < n < 12
    assert r["gbuf"][0, 7] == pytest.approx(acc, rel=1e-13)
    assert r["gbuf"][0, 15] == pytest.approx(T, rel=1e-13)


def test_stop_rule_ends_the_walk():
    """The walk ends at the first Gaussian that would take T below T_min: a
    faint Gaussian behind it, which alone would keep T above T_min, does not
    contribute. Opacities 0.98, 0.96 give T = 8e-4; 0.9 would give 8e-5 < 1e-4
    (stop); 0.05 behind it would give 7.6e-4."""
    pair = _pair_looking_down_z(W=8, H=8, fx=20.0)
    x = (4.5 - pair.cx) / pair.fx
    zs = [2.0, 2.2, 2.4, 2.6]
    ops = [0.98, 0.96, 0.9, 0.05]
    sc = _scene([[x * z, x * z, z] for z in zs], [[-1.0] * 3] * 4, [[1, 0, 0, 0]] * 4,
                [math.log(o / (1 - o)) for o in ops], rough=zs)
    r = O.render_pair(sc, pair, sg.mlp_spec(1, "basic", [8]), O.Cfg(dilation=0.0),
                      pixels=np.array([[4, 4]], np.int32), mlp_out=np.zeros((4, 4)))
    assert r["ncontrib"][0] == 2
    assert r["gbuf"][0, 15] == pytest.approx(0.02 * 0.04, rel=1e-12)
    assert r["gbuf"][0, 7] == pytest.approx(0.98 * 2.0 + 0.02 * 0.96 * 2.2, rel=1e-12)


# ---------------------------------------------------------------- BRDF (Eq. 4)

def test_brdf_normal_incidence_closed_form():
    n = np.array([0.0, 0.0, 1.0])
    base = np.array([0.7, 0.4, 0.2])
    for rough, metal in [(0.3, 0.0), (0.6, 0.5), (1.0, 1.0)]:
        fs, fd = O.brdf(n, n, n, base, rough, metal)
        a = rough ** 2
        F0 = 0.04 * (1 - metal) + base * metal
        assert np.allclose(fs, F0 / (4 * math.pi * a * a), rtol=1e-13)
        assert np.allclose(fd, (1 - metal) * base / math.pi, rtol=1e-14)


def test_brdf_rough_dielectric_at_sixty_degrees():
    """r = 1 (alpha_r = 1: D = 1/pi, Smith term = 1/((1+n.wo)(1+n.wi)))."""
    n = np.array([0.0, 0.0, 1.0])
    wi = np.array([math.sin(math.pi / 3), 0.0, math.cos(math.pi / 3)])
    fs, fd = O.brdf(n, n, wi, np.array([0.3, 0.3, 0.3]), 1.0, 0.0)
    vh = math.cos(math.pi / 6)
    F = 0.04 + 0.96 * (1 - vh) ** 5
    expect = (1 / math.pi) * F / ((1 + 1) * (1 + 0.5))
    assert np.allclose(fs, expect, rtol=1e-13)
    with open(os.path.join(GOLDEN, "closed_forms.json")) as fh:
        gold = json.load(fh)["brdf_rough_dielectric_60deg"]
    assert fs[0] == pytest.approx(gold["fs"], rel=1e-12)
    assert fd[0] == pytest.approx(gold["fd"], rel=1e-12)


def test_ggx_distribution_is_normalised():
    """int D(h) (n.h) dw_h = 1: recover D from f_s with F = 1 and w_o = w_i = h."""
    n = np.array([0.0, 0.0, 1.0])
    for rough in (0.3, 0.6, 0.9):
        a2 = rough ** 4
        th = np.linspace(0, math.pi / 2, 40001)
        Ds = []
        for t in th:
            h = np.array([math.sin(t), 0.0, math.cos(t)])
            fs, _ = O.brdf(n, h, h, np.ones(3), rough, 1.0)      # F0 = 1 => F = 1
            c = max(math.cos(t), 0.0)
            lam = c + math.sqrt(a2 + (1 - a2) * c * c)
            Ds.append(fs[0] * lam * lam)
        Ds = np.array(Ds)
        val = np.trapezoid(Ds * np.cos(th) * np.sin(th) * 2 * math.pi, th)
        assert val == pytest.approx(1.0, abs=2e-4)


def test_specular_directional_albedo_is_near_one_for_smooth_conductor():
    """White-furnace style: F = 1, w_o = n, int f_s (n.w_i) dw_i ~ 1 (slightly
    below: single-scattering GGX loses a little energy). A missing factor 4 or
    a squared visibility term moves this far from 1."""
    n = np.array([0.0, 0.0, 1.0])
    th = np.linspace(0, math.pi / 2, 60001)
    vals = []
    for t in th:
        wi = np.array([math.sin(t), 0.0, math.cos(t)])
        fs, _ = O.brdf(n, n, wi, np.ones(3), 0.3, 1.0)
        vals.append(fs[0])
    alb = np.trapezoid(np.array(vals) * np.cos(th) * np.sin(th) * 2 * math.pi, th)
    assert 0.97 < alb <= 1.0


# ---------------------------------------------------------------- deferred shading (Eq. 7)

def _gbuf_pixel(A, depth, n, base, rough, metal, sss, Ls, Lin):
    g = np.zeros(16)
    g[0] = A * depth
    g[1:4] = A * np.asarray(n)
    g[4:7] = A * np.asarray(base)
    g[7], g[8], g[9] = A * rough, A * metal, A * sss
    g[10:13] = A * np.asarray(Ls)
    g[13] = A * Lin
    g[15] = 1 - A
    return g


def test_deferred_position_and_blend_closed_forms():
    """Centre pixel of a camera at the origin looking along +z: the surface point
    at composited depth d is (0, 0, d). With the light and normal chosen, w_o, w_i
    and the BRDF are known, so Eq. 7 is checked end to end."""
    pair = _pair_looking_down_z(W=16, H=16, fx=30.0, light=(0.0, 3.0, 3.0))
    pair.cx = pair.cy = 8.5            # principal point on the centre of pixel (8, 8)
    d = 3.0
    x = np.array([0.0, 0.0, d])
    wo = -x / np.linalg.norm(x)
    wi = (pair.light - x) / np.linalg.norm(pair.light - x)
    n = np.array([0.0, 0.6, -0.8])
    base, rough, metal, Ls, Lin, A = [0.6, 0.5, 0.4], 0.7, 0.2, [0.3, 0.2, 0.1], 1.7, 0.8
    pix = np.array([[8, 8]], np.int32)
    fs, fd = O.brdf(n, wo, wi, np.array(base), rough, metal)
    ni = max(n @ wi, 0.0)
    for sss, expect in [(1.0, A * np.array(Ls)),
                        (0.0, A * (fs + fd) * Lin * ni),
                        (0.25, A * (0.25 * np.array(Ls) + 0.75 * (fs + fd) * Lin * ni))]:
        g = _gbuf_pixel(A, d, n, base, rough, metal, sss, Ls, Lin)[None, :]
        img, _ = O.shade(g, np.ones(1, np.int32), pix, pair)
        assert np.allclose(img[0], expect, rtol=1e-12)
    # no coverage => black
    img, _ = O.shade(np.zeros((1, 16)) + np.eye(16)[15], np.zeros(1, np.int32), pix, pair)
    assert np.all(img == 0)


# ---------------------------------------------------------------- MLP (Eq. 6)

def test_mlp_matches_torch_linear_chain_fp64():
    import torch
    spec = sg.mlp_spec(4, "pe6", [128, 128, 128, 128])
    rng = np.random.default_rng(0)
    X = rng.standard_normal((257, 64))
    _, y, Ls, Lin = O.mlp_forward(spec, X)
    layers = []
    for l, (W, b) in enumerate(zip(spec.weights, spec.biases)):
        lin = torch.nn.Linear(W.shape[1], W.shape[0]).double()
        with torch.no_grad():
            lin.weight.copy_(torch.from_numpy(W))
            lin.bias.copy_(torch.from_numpy(b))
        layers.append(lin)
        if l < len(spec.weights) - 1:
            layers.append(torch.nn.ReLU())
    net = torch.nn.Sequential(*layers)
    Xt = torch.from_numpy(X).requires_grad_(True)
    yt = net(Xt)
    assert np.allclose(yt.detach().numpy(), y, rtol=1e-12, atol=1e-12)
    assert np.allclose(torch.sigmoid(yt[:, :3]).detach().numpy(), Ls, rtol=1e-12)
    # backward through both heads vs autograd
    dLs = rng.standard_normal((257, 3))
    dLin = rng.standard_normal(257)
    acts, y2, Ls2, _ = O.mlp_forward(spec, X)
    dWs, dbs, dX = O.mlp_backward(spec, acts, y2, Ls2, dLs, dLin)
    out = (torch.sigmoid(yt[:, :3]) * torch.from_numpy(dLs)).sum() + \
        (torch.relu(yt[:, 3]) * torch.from_numpy(dLin)).sum()
    out.backward()
    assert np.allclose(Xt.grad.numpy(), dX, rtol=1e-10, atol=1e-12)
    for l, lin in enumerate([m for m in net if isinstance(m, torch.nn.Linear)]):
        assert np.allclose(lin.weight.grad.numpy(), dWs[l], rtol=1e-10, atol=1e-12)
        assert np.allclose(lin.bias.grad.numpy(), dbs[l], rtol=1e-10, atol=1e-12)


def test_bf16_rounding_matches_torch_bfloat16():
    import torch
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-6, 6, 20000),
                        np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8), 0.0])])
    x32 = x.astype(np.float32).astype(np.float64)        # torch converts from float32
    ref = torch.from_numpy(x32).float().bfloat16().double().numpy()
    assert np.array_equal(O.bf16_round(x32), ref)


def test_input_encoding_gradients_match_autograd():
    import torch
    import math as m
    wl = sg.make_workload("c3", N=50, res=32)
    sc, pair = wl.scenes[0], wl.pairs[0]
    dX = np.random.default_rng(2).standard_normal((50, 64))
    dmu, dn, dv = O.input_grads("pe6", dX, sc.mu, pair.center, pair.light)
    mu = torch.from_numpy(sc.mu).requires_grad_(True)
    nn_ = torch.from_numpy(sc.normal).requires_grad_(True)
    vv = torch.from_numpy(sc.vis).requires_grad_(True)
    C = torch.from_numpy(pair.center)
    Lp = torch.from_numpy(pair.light)
    feats = []
    for k in range(6):
        feats += [torch.sin((2.0 ** k) * m.pi * mu), torch.cos((2.0 ** k) * m.pi * mu)]
    wo = (C - mu) / (C - mu).norm(dim=1, keepdim=True)
    wi = (Lp - mu) / (Lp - mu).norm(dim=1, keepdim=True)
    X = torch.cat(feats + [mu, wo, wi, nn_, (Lp - mu).norm(dim=1, keepdim=True), vv[:, None],
                           torch.zeros(50, 14, dtype=torch.float64)], 1)
    assert np.allclose(X.detach().numpy(), O.mlp_inputs("pe6", sc.mu, sc.normal, sc.vis,
                                                        pair.center, pair.light), atol=1e-14)
    (X * torch.from_numpy(dX)).sum().backward()
    assert np.allclose(mu.grad.numpy(), dmu, rtol=1e-11, atol=1e-12)
    assert np.allclose(nn_.grad.numpy(), dn)
    assert np.allclose(vv.grad.numpy(), dv)


def _paper_torch(spec):
    """The paper's network (App. E "Network") assembled from torch.nn modules."""
    import torch

    def lin(W, b):
        m = torch.nn.Linear(W.shape[1], W.shape[0]).double()
        with torch.no_grad():
            m.weight.copy_(torch.from_numpy(np.asarray(W, np.float64)))
            m.bias.copy_(torch.from_numpy(np.asarray(b, np.float64)))
        return m

    L = [lin(W, b) for W, b in zip(spec.weights, spec.biases)]
    act = torch.nn.LeakyReLU(O.LRELU_SLOPE)
    trunk = torch.nn.Sequential(L[0], act, L[1], act, L[2], act)
    incident = torch.nn.Sequential(L[3], act, L[4], torch.nn.ReLU())
    sss = torch.nn.Sequential(L[5], torch.nn.Sigmoid())
    return L, trunk, incident, sss


def test_paper_mlp_matches_torch_modules_fp64():
    import torch
    spec = sg.mlp_spec(6, "paper", [])
    rng = np.random.default_rng(3)
    X = rng.standard_normal((300, 48))
    acts, y, Ls, Lin = O.mlp_forward(spec, X)
    L, trunk, incident, sss = _paper_torch(spec)
    Xt = torch.from_numpy(X).requires_grad_(True)
    t = trunk(Xt)
    Lin_t, Ls_t = incident(t)[:, 0], sss(t)
    assert np.allclose(Ls_t.detach().numpy(), Ls, rtol=1e-12, atol=1e-14)
    assert np.allclose(Lin_t.detach().numpy(), Lin, rtol=1e-12, atol=1e-14)
    dLs = rng.standard_normal((300, 3))
    dLin = rng.standard_normal(300)
    dWs, dbs, dX = O.mlp_backward(spec, acts, y, Ls, dLs, dLin)
    ((Ls_t * torch.from_numpy(dLs)).sum() + (Lin_t * torch.from_numpy(dLin)).sum()).backward()
    assert np.allclose(Xt.grad.numpy(), dX, rtol=1e-10, atol=1e-12)
    for l, m in enumerate(L):
        assert np.allclose(m.weight.grad.numpy(), dWs[l], rtol=1e-10, atol=1e-12), l
        assert np.allclose(m.bias.grad.numpy(), dbs[l], rtol=1e-10, atol=1e-12), l


def test_paper_input_encoding_and_gradients_match_autograd():
    import math as m
    import torch
    wl = sg.make_workload("c3", N=60, res=32, net="paper")
    sc, pair = wl.scenes[0], wl.pairs[0]
    dX = np.random.default_rng(5).standard_normal((60, 48))
    dmu, dn, dv, dq, dls = O.input_grads("paper", dX, sc.mu, pair.center, pair.light, sc.quat, sc.log_s)
    mu = torch.from_numpy(sc.mu.astype(np.float64)).requires_grad_(True)
    nn_ = torch.from_numpy(sc.normal.astype(np.float64)).requires_grad_(True)
    vv = torch.from_numpy(sc.vis.astype(np.float64)).requires_grad_(True)
    q = torch.from_numpy(sc.quat.astype(np.float64)).requires_grad_(True)
    ls = torch.from_numpy(sc.log_s.astype(np.float64)).requires_grad_(True)
    C, Lp = torch.from_numpy(pair.center), torch.from_numpy(pair.light)
    wo = (C - mu) / (C - mu).norm(dim=1, keepdim=True)
    wi = (Lp - mu) / (Lp - mu).norm(dim=1, keepdim=True)
    feats = [nn_, q / q.norm(dim=1, keepdim=True), torch.exp(ls), wi, wo,
             (Lp - mu).norm(dim=1, keepdim=True), vv[:, None]]
    for k in range(4):
        feats += [torch.sin((2.0 ** k) * m.pi * mu), torch.cos((2.0 ** k) * m.pi * mu)]
    X = torch.cat(feats + [torch.zeros(60, 6, dtype=torch.float64)], 1)
    assert np.allclose(X.detach().numpy(), O.mlp_inputs("paper", sc.mu, sc.normal, sc.vis, pair.center,
                                                        pair.light, sc.quat, sc.log_s), atol=1e-14)
    (X * torch.from_numpy(dX)).sum().backward()
    for got, ref in [(dmu, mu), (dn, nn_), (dv, vv), (dq, q), (dls, ls)]:
        assert np.allclose(ref.grad.numpy(), got, rtol=1e-11, atol=1e-12)


# ---------------------------------------------------------------- training losses (App. E "Losses")

def test_ssim_equals_brute_force_window_sums():
    """Separable windowed moments == explicit 11 x 11 window sums with zero
    padding, pixel by pixel (tiny image)."""
    rng = np.random.default_rng(11)
    H, W = 9, 12
    x, y = rng.uniform(0, 1, (H, W, 3)), rng.uniform(0, 1, (H, W, 3))
    w1 = O.losses.gaussian_window()
    w2 = np.outer(w1, w1)
    S = np.zeros((H, W, 3))
    for i in range(H):
        for j in range(W):
            acc = np.zeros((5, 3))
            for a in range(-5, 6):
                for b in range(-5, 6):
                    ii, jj = i + a, j + b
                    if 0 <= ii < H and 0 <= jj < W:
                        wt = w2[a + 5, b + 5]
                        xv, yv = x[ii, jj], y[ii, jj]
                        acc += wt * np.stack([xv, yv, xv * xv, yv * yv, xv * yv])
            mx, my, exx, eyy, exy = acc
            sx, sy, sxy = exx - mx * mx, eyy - my * my, exy - mx * my
            C1, C2 = O.losses.SSIM_C1, O.losses.SSIM_C2
            S[i, j] = (2 * mx * my + C1) * (2 * sxy + C2) / ((mx * mx + my * my + C1) * (sx + sy + C2))
    assert np.allclose(O.ssim_map(x, y), S, rtol=1e-12, atol=1e-14)
    assert np.isclose(O.ssim(x, y)[0], S.mean(), rtol=1e-12)


def test_ssim_closed_forms():
    rng = np.random.default_rng(12)
    x = rng.uniform(0, 1, (20, 24, 3))
    assert np.isclose(O.ssim(x, x)[0], 1.0, atol=1e-12)
    c, d = 0.3, 0.7                      # constant images: interior S = (2cd + C1) / (c^2 + d^2 + C1)
    S = O.ssim_map(np.full((20, 24, 3), c), np.full((20, 24, 3), d))
    C1 = O.losses.SSIM_C1
    assert np.allclose(S[5:-5, 5:-5], (2 * c * d + C1) / (c * c + d * d + C1), rtol=1e-12)


def test_image_and_incident_loss_gradients_match_finite_differences():
    rng = np.random.default_rng(13)
    x, y = rng.uniform(0, 1, (10, 13, 3)), rng.uniform(0, 1, (10, 13, 3))
    loss, g = O.image_loss(x, y)
    for _ in range(12):
        i, j, c = rng.integers(10), rng.integers(13), rng.integers(3)
        h = 1e-6
        xp, xm = x.copy(), x.copy()
        xp[i, j, c] += h
        xm[i, j, c] -= h
        fd = (O.image_loss(xp, y)[0] - O.image_loss(xm, y)[0]) / (2 * h)
        assert abs(fd - g[i, j, c]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (fd, g[i, j, c])
    L_in = np.array([0.2, 1.5, 0.7, 0.95])
    v = np.array([0.5, 0.1, 0.7 - 0.25, 0.95 + 0.01])
    val, dl, dv = O.incident_loss(L_in, v)
    assert np.isclose(val, 0.02 * (0.3 + 0.9 + 0.25 + 0.01) / 4)
    assert np.allclose(dl, 0.02 / 4 * np.array([-1, 0, 1, -1]))     # clamped entry: no gradient to L_in
    assert np.allclose(dv, -0.02 / 4 * np.array([-1, 1, 1, -1]))


def test_ssim_and_image_loss_gradients_equal_conv2d_autograd():
    """SSIM with torch's conv2d (11 x 11 Gaussian window, zero padding) in
    FP64 and autograd: the oracle's SSIM, image loss and their gradients,
    every entry of a ragged 13 x 17 image."""
    import torch
    import torch.nn.functional as Fn
    rng = np.random.default_rng(21)
    x, y = rng.uniform(0, 1, (13, 17, 3)), rng.uniform(0, 1, (13, 17, 3))
    w1 = torch.from_numpy(O.losses.gaussian_window())
    win = (w1[:, None] * w1[None, :]).expand(3, 1, 11, 11).contiguous()
    xt = torch.from_numpy(x).permute(2, 0, 1)[None].clone().requires_grad_(True)
    yt = torch.from_numpy(y).permute(2, 0, 1)[None]
    wm = lambda a: Fn.conv2d(a, win, padding=5, groups=3)
    mx, my = wm(xt), wm(yt)
    sxx, syy, sxy = wm(xt * xt) - mx * mx, wm(yt * yt) - my * my, wm(xt * yt) - mx * my
    C1, C2 = O.losses.SSIM_C1, O.losses.SSIM_C2
    S = ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))
    lam = 0.2
    loss = (1 - lam) * (xt - yt).abs().mean() + lam * (1 - S.mean())
    loss.backward()
    s_val, _ = O.ssim(x, y)
    l_val, g = O.image_loss(x, y, lam)
    assert s_val == pytest.approx(float(S.mean().detach()), rel=1e-13)
    assert l_val == pytest.approx(float(loss.detach()), rel=1e-13)
    np.testing.assert_allclose(g, xt.grad[0].permute(1, 2, 0).numpy(), rtol=1e-10, atol=1e-14)


# ---------------------------------------------------------------- binning / sort

def test_bin_sort_equals_python_stable_sort():
    P, N, tx, ty = 3, 400, 7, 5
    rect, depth = sg.synthetic_bin_inputs(9, P, N, tx, ty)
    dkey = depth.view(np.uint32)
    item_pair = np.repeat(np.arange(P), N)
    tiles_x = np.full(P, tx)
    tile_off = np.arange(P) * tx * ty
    n, keys, vals, ranges = O.bin_sort(item_pair, rect, dkey, tiles_x, tile_off, P * tx * ty)
    inst = []
    for m in range(P * N):
        x0, x1, y0, y1 = rect[m]
        for yy in range(y0, y1 + 1):
            for xx in range(x0, x1 + 1):
                inst.append((int(tile_off[item_pair[m]] + yy * tx + xx), int(dkey[m]), m))
    inst.sort()                           # Python's stable sort on the tuple
    assert n == len(inst)
    assert list(keys) == [t for t, _, _ in inst]
    assert list(vals) == [m for _, _, m in inst]
    for t in range(P * tx * ty):
        sel = [i for i, (tt, _, _) in enumerate(inst) if tt == t]
        if sel:
            assert tuple(ranges[t]) == (sel[0], sel[-1] + 1)
        else:
            assert tuple(ranges[t]) == (0, 0)
