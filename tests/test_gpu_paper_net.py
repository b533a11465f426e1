"""The paper's network (App. E "Network"; kind SSSGS_MLP_PAPER) on the GPU,
through the C ABI, against the FP64 oracle.

* network alone: outputs, the six weight/bias gradients and the 14 input
  gradients per item (mu, n, v, quat, log_s) for a seeded upstream gradient;
* whole step: image and every scene / network gradient, with the network's
  rotation and scale inputs adding to the projection's quat and log_s
  gradients;
* the BF16 tensor-core path does not take this network: it reports
  SSSGS_ERR_UNSUPPORTED instead of running something else.
"""
import numpy as np
import pytest
import torch

import oracle as O
import scenegen as sg
from gpu_common import assert_grads_close, assert_image_close, flagged, oracle_batch, run_gpu
from paper_2408_12282_gb300 import binding as B
from paper_2408_12282_gb300 import pipeline as PL

pytestmark = pytest.mark.gpu

SCENE_KEYS = PL.SCENE_KEYS


@pytest.fixture(scope="module", autouse=True)
def _lib(gpu_lib):
    return gpu_lib


def _rel(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def _network_only_check(wl, tol, seed=17):
    """mlp_fwd, then mlp_bwd with a seeded upstream gradient, against the
    oracle's network: outputs, every weight/bias gradient, the input gradients."""
    kind = wl.mlp.kind
    r = PL.renderer_for_workload(wl, precision=B.FP32)
    t = r.table
    B.mlp_fwd(r._mlp_s, t.h, t.d, r._scene_s, r.mlp_out, r.status)
    n = t.n_items
    up = np.random.default_rng(seed).uniform(-1, 1, (n, 4)).astype(np.float32)
    r.zero_grads()
    r.drec[:, 16:20] = torch.from_numpy(up).cuda()
    r.dx_items.fill_(float("nan"))
    B.mlp_bwd(r._mlp_s, t.h, t.d, r._scene_s, r.drec, r._mlp_g, r.dx_items, r.ws_mlp, r.status)
    torch.cuda.synchronize()
    out = r.mlp_out.double().cpu().numpy()
    dx = r.dx_items.double().cpu().numpy()
    dW = [w.double().cpu().numpy() for w in r.dW]
    db = [b.double().cpu().numpy() for b in r.db]
    nl = len(dW)
    rdW = [np.zeros_like(w) for w in dW]
    rdb = [np.zeros_like(b) for b in db]
    rdx = np.zeros_like(dx)
    off = 0
    for pair in wl.pairs:
        sc = wl.scenes[pair.scene]
        X = O.mlp_inputs(kind, sc.mu, sc.normal, sc.vis, pair.center, pair.light, sc.quat, sc.log_s)
        acts, y, Ls, Lin = O.mlp_forward(wl.mlp, X)
        np.testing.assert_allclose(out[off:off + sc.N, :3], Ls, atol=2e-6)
        np.testing.assert_allclose(out[off:off + sc.N, 3], Lin, atol=2e-5 * max(1.0, np.abs(Lin).max()))
        u = up[off:off + sc.N].astype(np.float64)
        gW, gb, gX = O.mlp_backward(wl.mlp, acts, y, Ls, u[:, :3], u[:, 3])
        for l in range(nl):
            rdW[l] += gW[l]
            rdb[l] += gb[l]
        gi = O.input_grads(kind, gX, sc.mu, pair.center, pair.light, sc.quat, sc.log_s)
        rdx[off:off + sc.N, 0:3] = gi[0]
        rdx[off:off + sc.N, 3:6] = gi[1]
        rdx[off:off + sc.N, 6] = gi[2]
        if kind == "paper":
            rdx[off:off + sc.N, 7:11] = gi[3]
            rdx[off:off + sc.N, 11:14] = gi[4]
        off += sc.N
    assert np.isfinite(dx).all()
    errs = {f"W{l}": _rel(dW[l], rdW[l]) for l in range(nl)}
    errs.update({f"b{l}": _rel(db[l], rdb[l]) for l in range(nl)})
    errs.update({"dmu": _rel(dx[:, 0:3], rdx[:, 0:3]), "dn": _rel(dx[:, 3:6], rdx[:, 3:6]),
                 "dv": _rel(dx[:, 6], rdx[:, 6])})
    if kind == "paper":
        errs.update({"dq": _rel(dx[:, 7:11], rdx[:, 7:11]), "dlog_s": _rel(dx[:, 11:14], rdx[:, 11:14])})
    else:
        assert not dx[:, 7:].any()
    print(f"\n{kind} network FP32 rel-L2:", {k: f"{v:.1e}" for k, v in errs.items()})
    assert all(v < tol for v in errs.values()), errs


def test_paper_network_forward_and_backward_match_oracle():
    _network_only_check(sg.make_workload("c4", N=3000, res=64, n_pairs=3, net="paper"), 1e-4)


def test_chain_network_any_width_multiple_of_16():
    """Hidden widths 48, 96, 80 (every multiple of 16 up to 128 has a
    register-tiled form in the CUDA-core network)."""
    wl = sg.make_workload("c1")
    wl.mlp = sg.mlp_spec(21, "basic", [48, 96, 80])
    _network_only_check(wl, 1e-4)


def test_paper_network_whole_step_image_and_gradients():
    wl = sg.make_workload("c2", N=20000, res=128, net="paper")
    ref0 = oracle_batch(wl, [0])
    fl = flagged(ref0["margin"])
    dimg = sg.random_dimg(41, ref0["img"].shape[0])
    dimg[fl] = 0.0
    ref = oracle_batch(wl, [0], dimg=dimg)
    g = run_gpu(wl, precision=B.FP32, dimg=dimg)
    assert_image_close(g["img"], ref0["img"], fl)
    assert_grads_close(g["grads"], ref["grads"], SCENE_KEYS)
    errs = {f"W{l}": _rel(g["dW"][l], ref["dW"][l]) for l in range(6)}
    errs.update({f"b{l}": _rel(g["db"][l], ref["db"][l]) for l in range(6)})
    print("\npaper network step, weight gradients rel-L2:", {k: f"{v:.1e}" for k, v in errs.items()})
    assert all(v < 1e-3 for v in errs.values()), errs


def test_paper_network_has_no_bf16_path():
    wl = sg.make_workload("c1", net="paper")
    r = PL.renderer_for_workload(wl, precision=B.BF16)
    t = r.table
    with pytest.raises(B.SSSGSError, match=str(-3)):
        B.mlp_fwd(r._mlp_s, t.h, t.d, r._scene_s, r.mlp_out, r.status)
