"""The produced gradients train: Adam on the scene parameters through the
torch.autograd.Function (SSSRenderFunction) reduces the L1 loss to a target
rendered from perturbed parameters (the c1 recipe)."""
import pytest
import torch

import scenegen as sg
from paper_2408_12282_gb300 import binding as B
from paper_2408_12282_gb300 import pipeline as PL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib(gpu_lib):
    return gpu_lib


@pytest.mark.parametrize("shading", ["deferred", "gaussian"])
def test_adam_steps_reduce_the_l1_loss(shading):
    wl = sg.make_workload("c1", N=1024, res=64)
    wl_t = sg.Workload(wl.name, [wl.target_scene], wl.pairs, wl.mlp, wl.tile)
    rt = PL.renderer_for_workload(wl_t, shading=shading)
    rt.fit_capacity()
    rt.forward()
    target = rt.img.clone()
    r = PL.renderer_for_workload(wl, shading=shading)
    r.fit_capacity(2.0)
    params = [r.scene[k] for k in ("mu", "log_s", "base", "logit_o")]
    for p in params:
        p.requires_grad_(True)
    opt = torch.optim.Adam(params, lr=2e-3)
    losses = []
    for _ in range(40):
        opt.zero_grad()
        img = PL.render(r)
        loss = (img - target).abs().mean()
        loss.backward()
        opt.step()
        r.check_status()
        losses.append(loss.item())
    print(f"\n{shading}: L1 {losses[0]:.5f} -> {losses[-1]:.5f}")
    assert losses[-1] < 0.7 * losses[0]
