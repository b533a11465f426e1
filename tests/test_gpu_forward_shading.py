"""Per-Gaussian shading (the paper's "w/o Deferred" ablation) on the GPU,
through the C ABI, against the oracle's render_pair(per_gaussian_shading=True):
image and every scene and network gradient (flagged pixels excluded and given
zero upstream gradient, as in the deferred-path tests)."""
import numpy as np
import pytest
import torch

import oracle as O
import scenegen as sg
from gpu_common import assert_grads_close, assert_image_close, flagged
from paper_2408_12282_gb300 import binding as B
from paper_2408_12282_gb300 import pipeline as PL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib(gpu_lib):
    return gpu_lib


def _rel(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("name,kw", [("c1", dict(N=1024, res=64)), ("c2", dict(N=20000, res=96)),
                                     ("c2", dict(N=20000, res=96, net="paper"))])
def test_per_gaussian_shading_matches_oracle(name, kw):
    wl = sg.make_workload(name, **kw)
    pair, sc = wl.pairs[0], wl.scenes[0]
    ref0 = O.render_pair(sc, pair, wl.mlp, O.Cfg(tile=wl.tile), per_gaussian_shading=True)
    fl = flagged(ref0["margin"])
    dimg = sg.random_dimg(31, ref0["img"].shape[0])
    dimg[fl] = 0.0
    ref = O.render_pair(sc, pair, wl.mlp, O.Cfg(tile=wl.tile), dimg=dimg, per_gaussian_shading=True)
    r = PL.renderer_for_workload(wl, precision=B.FP32, shading="gaussian")
    r.fit_capacity()
    r.forward()
    r.backward(dimg=torch.from_numpy(np.ascontiguousarray(dimg, np.float32)).cuda())
    torch.cuda.synchronize()
    r.check_status()
    assert_image_close(r.img.double().cpu().numpy(), ref0["img"], fl)
    got = {k: v.double().cpu().numpy() for k, v in r.grads.items()}
    rep = assert_grads_close(got, ref["grads"], PL.SCENE_KEYS)
    errs = {f"W{l}": _rel(r.dW[l].cpu().numpy(), ref["dW"][l]) for l in range(len(ref["dW"]))}
    print(f"\n{name} {kw}: per-Gaussian shading, {int(fl.sum())} flagged px; grads",
          {k: f"{v[0]:.1e}" for k, v in rep.items()}, "net", {k: f"{v:.1e}" for k, v in errs.items()})
    assert all(v < 1e-3 for v in errs.values()), errs


def test_per_gaussian_shading_with_the_paper_losses_runs():
    """loss='paper' (image loss + incident constraint) on the per-Gaussian path:
    the image-loss gradient feeds the same backward."""
    wl = sg.make_workload("c2", N=8000, res=64)
    r = PL.renderer_for_workload(wl, precision=B.FP32, shading="gaussian")
    r.fit_capacity()
    r.forward()
    target = torch.rand_like(r.img)
    r.backward(target=target, loss="paper")
    torch.cuda.synchronize()
    assert float(r.loss[0]) > 0 and torch.isfinite(r.grads["mu"]).all() and r.grads["base"].abs().sum() > 0
