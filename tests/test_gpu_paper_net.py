"""The paper's network (App. E "Network"; kind SSSGS_MLP_PAPER) on the GPU,
through the C ABI, against the FP64 oracle.

* network alone: outputs, the six weight/bias gradients and the 14 input
  gradients per item (mu, n, v, quat, log_s) for a seeded upstream gradient;
* whole step: image and every scene / network gradient, with the network's
  rotation and scale inputs adding to the projection's quat and log_s
  gradients;
* the BF16 tensor-core kernels (mlp_tc_paper.cu): forward and backward
  against the oracle's BF16-emulating network.
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


@pytest.mark.parametrize("N,n_pairs", [(3000, 3), (20000, 2)])
def test_paper_network_bf16_forward_matches_bf16_oracle(N, n_pairs):
    """Tensor-core forward vs the oracle's BF16-emulating network, with the
    gates of the other BF16 network (bf16 rounding flips of hidden units)."""
    wl = sg.make_workload("c4", N=N, res=64, n_pairs=n_pairs, net="paper")
    r = PL.renderer_for_workload(wl, precision=B.BF16)
    t = r.table
    B.mlp_fwd(r._mlp_s, t.h, t.d, r._scene_s, r.mlp_out, r.status)
    torch.cuda.synchronize()
    r.check_status()
    got = r.mlp_out.double().cpu().numpy()
    ref = []
    for pair in wl.pairs:
        sc = wl.scenes[pair.scene]
        X = O.mlp_inputs("paper", sc.mu, sc.normal, sc.vis, pair.center, pair.light, sc.quat, sc.log_s)
        _, _, Ls, Lin = O.mlp_forward(wl.mlp, X, bf16=True)
        ref.append(np.concatenate([Ls, Lin[:, None]], 1))
    err = np.abs(got - np.concatenate(ref))
    print(f"\npaper net bf16 N={N}: max {err.max():.3e} mean {err.mean():.3e} frac>1e-4 {(err > 1e-4).mean():.4f}")
    assert (err > 1e-4).mean() < 0.01
    assert err.max() < 2e-2
    assert err.mean() < 1e-4


@pytest.mark.parametrize("N,n_pairs,zero_frac", [(3000, 3, 0.0), (20000, 2, 0.0), (20000, 2, 0.6)])
def test_paper_network_bf16_backward_matches_bf16_oracle(N, n_pairs, zero_frac):
    """Tensor-core backward (runs on the rows with a nonzero upstream
    gradient) vs the BF16-emulating oracle. At >= 40K rows per tensor rel-L2
    <= 2e-3, input gradients <= 3e-3 (measured: weights and biases at most
    1.5e-3, inputs 1.9e-3; the narrow 32-unit layers with Leaky-ReLU give
    each flipped bf16 decision more weight than the 128-unit network, whose
    gate is 1e-3); with fewer rows at most 0.1% of rows off by > 1e-2
    relative and rel-L2 <= 1e-2. Rows with a zero upstream gradient must get
    exactly zero input gradients."""
    wl = sg.make_workload("c4", N=N, res=64, n_pairs=n_pairs, net="paper")
    r = PL.renderer_for_workload(wl, precision=B.BF16)
    n = r.table.n_items
    rng = np.random.default_rng(N + 1)
    up = rng.uniform(-1, 1, (n, 4)).astype(np.float32)
    zero = rng.uniform(size=n) < zero_frac
    up[zero] = 0.0
    r.zero_grads()
    r.drec[:, 16:20] = torch.from_numpy(up).cuda()
    r.dx_items.fill_(float("nan"))
    t = r.table
    B.mlp_bwd(r._mlp_s, t.h, t.d, r._scene_s, r.drec, r._mlp_g, r.dx_items, r.ws_mlp, r.status)
    torch.cuda.synchronize()
    r.check_status()
    dW = [w.double().cpu().numpy() for w in r.dW]
    db = [b.double().cpu().numpy() for b in r.db]
    dx = r.dx_items.double().cpu().numpy()
    rdW = [np.zeros_like(w) for w in dW]
    rdb = [np.zeros_like(b) for b in db]
    rdx = np.zeros_like(dx)
    off = 0
    for pair in wl.pairs:
        sc = wl.scenes[pair.scene]
        X = O.mlp_inputs("paper", sc.mu, sc.normal, sc.vis, pair.center, pair.light, sc.quat, sc.log_s)
        acts, y, Ls, Lin = O.mlp_forward(wl.mlp, X, bf16=True)
        u = up[off:off + sc.N].astype(np.float64)
        gW, gb, gX = O.mlp_backward(wl.mlp, acts, y, Ls, u[:, :3], u[:, 3], bf16=True)
        for l in range(6):
            rdW[l] += gW[l]
            rdb[l] += gb[l]
        dmu, dn, dv, dq, dls = O.input_grads("paper", gX, sc.mu, pair.center, pair.light, sc.quat, sc.log_s)
        rdx[off:off + sc.N] = np.concatenate([dmu, dn, dv[:, None], dq, dls], 1)
        off += sc.N
    assert np.all(dx[zero] == 0.0) and np.isfinite(dx).all()
    errs = {f"W{l}": _rel(dW[l], rdW[l]) for l in range(6)}
    errs.update({f"b{l}": _rel(db[l], rdb[l]) for l in range(6)})
    errs["dx"] = _rel(dx, rdx)
    row_rel = np.abs(dx - rdx).max(1) / np.maximum(np.abs(rdx).max(1), 1e-12)
    frac_bad = float((row_rel > 1e-2).mean())
    print("\npaper net bf16 backward rel-L2:", {k: f"{v:.2e}" for k, v in errs.items()},
          f"rows >1e-2: {frac_bad:.4%}")
    if int((~zero).sum()) >= 40000:
        assert all(v < (3e-3 if k == "dx" else 2e-3) for k, v in errs.items()), errs
    else:
        assert frac_bad <= 1e-3
        assert all(v < 1e-2 for v in errs.values()), errs
