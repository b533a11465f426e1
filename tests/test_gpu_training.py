"""The produced gradients train: Adam on the scene parameters through the
torch.autograd.Function (SSSRenderFunction) reduces the L1 loss to a target
rendered from perturbed parameters (the c1 recipe); a checkpoint restores a
step exactly."""
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


def test_checkpoint_resume_replays_the_same_step(tmp_path):
    """Save the trainable state, change it, restore it: the captured graph
    (which reads the same buffers) renders the saved state's image again,
    bit for bit, and the same gradients up to atomic summation order."""
    wl = sg.make_workload("c4", N=4000, res=64, n_pairs=4)
    r = PL.renderer_for_workload(wl, precision=B.BF16)
    r.fit_capacity()
    target = torch.zeros(r.table.n_pixels, 3, device="cuda")
    graph = r.capture(target=target, l1_scale=1.0 / (3.0 * r.table.n_pixels))
    graph.replay()
    torch.cuda.synchronize()
    img0 = r.img.clone()
    g0 = {k: v.clone() for k, v in r.grads.items()}
    PL.save_checkpoint(tmp_path / "ck.pt", r, step=7)
    with torch.no_grad():
        r.scene["base"].mul_(0.5)
        r.mlp.W[0].mul_(1.1)
    graph.replay()
    torch.cuda.synchronize()
    assert not torch.equal(r.img, img0)
    assert PL.load_checkpoint(tmp_path / "ck.pt", r)["step"] == 7
    graph.replay()
    torch.cuda.synchronize()
    r.check_status()
    assert torch.equal(r.img, img0)
    for k, v in g0.items():
        assert torch.allclose(r.grads[k], v, rtol=1e-5, atol=1e-7 * float(v.abs().max()) + 1e-30), k
