"""The seeded input generators: every workload is a pure function of its
name, sizes and seed (both sides of every parity test draw the same inputs),
and the values are float32-representable (the CUDA path computes in FP32)."""
import numpy as np
import pytest

import scenegen as sg


def _arrays(wl):
    out = []
    for s in wl.scenes:
        out += [np.asarray(v) for v in s.arrays().values()]
    for p in wl.pairs:
        out += [np.asarray(p.R), np.asarray(p.t), np.asarray(p.light), np.array([p.fx, p.fy, p.cx, p.cy, p.W, p.H])]
    out += [np.asarray(w) for w in wl.mlp.weights] + [np.asarray(b) for b in wl.mlp.biases]
    return out


@pytest.mark.parametrize("name,kw", [("c1", {}), ("c4", dict(N=2000, res=32, n_pairs=3)),
                                     ("c5", dict(N=20000, res=32, n_pairs=2)),
                                     ("c6", dict(N=2000, res=32, n_views=2, n_lights=4))])
def test_workloads_are_deterministic_and_float32_exact(name, kw):
    a, b = _arrays(sg.make_workload(name, **kw)), _arrays(sg.make_workload(name, **kw))
    assert len(a) == len(b)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    for s in sg.make_workload(name, **kw).scenes:
        for v in s.arrays().values():
            v = np.asarray(v, np.float64)
            assert np.array_equal(v, v.astype(np.float32).astype(np.float64))


def test_seed_offset_changes_the_scene():
    a = sg.make_workload("c4", N=2000, res=32, n_pairs=2)
    b = sg.make_workload("c4", N=2000, res=32, n_pairs=2, seed_offset=1)
    assert not np.array_equal(a.scenes[0].mu, b.scenes[0].mu)


def test_dimg_and_sh_coefficients_are_seeded():
    assert np.array_equal(sg.random_dimg(3, 100), sg.random_dimg(3, 100))
    assert not np.array_equal(sg.random_dimg(3, 100), sg.random_dimg(4, 100))
    assert np.array_equal(sg.vis_sh_coeffs(2, 50), sg.vis_sh_coeffs(2, 50))
