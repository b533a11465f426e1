"""BF16 tensor-core network (tcgen05) vs the oracle's BF16-emulating network.

Both sides round the network input, the weights and every hidden activation
to bfloat16 (round to nearest even) and accumulate in higher precision (FP32
on the GPU, FP64 in the oracle). A hidden value whose FP64 and FP32 sums fall
on different sides of a bfloat16 rounding boundary rounds differently (one
bf16 ulp, 2^-8 relative); such flips are rare and their effect on the output
is bounded by a few bf16 ulps of a hidden unit times a weight. The gate:
  * 99% of outputs within 1e-4 of the oracle,
  * every output within 2e-2 (a handful of flips),
  * and the mean error far below the bf16 ulp of the inputs.
The error against the pure FP64 network is reported, not gated.
"""
import numpy as np
import pytest
import torch

import oracle as O
import scenegen as sg
from paper_2408_12282_gb300 import binding as B
from paper_2408_12282_gb300 import pipeline as PL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib(gpu_lib):
    return gpu_lib


def _gpu_mlp_out(wl, precision):
    r = PL.renderer_for_workload(wl, precision=precision)
    t = r.table
    B.mlp_fwd(r._mlp_s, t.h, t.d, r._scene_s, r.mlp_out, r.status)
    torch.cuda.synchronize()
    r.check_status()
    return r.mlp_out.double().cpu().numpy()


@pytest.mark.parametrize("N,n_pairs", [(3000, 3), (20000, 2)])
def test_bf16_network_forward_matches_bf16_oracle(N, n_pairs):
    wl = sg.make_workload("c4", N=N, res=64, n_pairs=n_pairs)
    got = _gpu_mlp_out(wl, B.BF16)
    ref_b, ref_f = [], []
    for pair in wl.pairs:
        sc = wl.scenes[pair.scene]
        X = O.mlp_inputs(wl.mlp.kind, sc.mu, sc.normal, sc.vis, pair.center, pair.light)
        _, _, Ls, Lin = O.mlp_forward(wl.mlp, X, bf16=True)
        ref_b.append(np.concatenate([Ls, Lin[:, None]], 1))
        _, _, Ls, Lin = O.mlp_forward(wl.mlp, X, bf16=False)
        ref_f.append(np.concatenate([Ls, Lin[:, None]], 1))
    ref_b = np.concatenate(ref_b)
    ref_f = np.concatenate(ref_f)
    err = np.abs(got - ref_b)
    err64 = np.abs(got - ref_f)
    print(f"\nbf16 net N={N}: vs bf16 oracle max {err.max():.3e} mean {err.mean():.3e} "
          f"frac>1e-4 {(err > 1e-4).mean():.4f}; vs fp64 max {err64.max():.3e} mean {err64.mean():.3e}")
    assert (err > 1e-4).mean() < 0.01
    assert err.max() < 2e-2
    assert err.mean() < 1e-4


def _rel(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("N,n_pairs,zero_frac", [(3000, 3, 0.0), (20000, 2, 0.0), (20000, 2, 0.6)])
def test_bf16_network_backward_matches_bf16_oracle(N, n_pairs, zero_frac):
    """Upstream dL/d(L_SSS, L_in) fixed (seeded); weight, bias and per-item
    input gradients of the tensor-core backward vs the BF16-emulating oracle.

    Besides bf16 rounding flips, a ReLU mask can differ: a pre-activation
    within ~1e-4 of zero (relative to the layer) changes sign when an
    upstream bf16 rounding flips, which changes that row's gradient by a
    finite amount. Re-running the oracle's bf16 network with FP32 instead of
    FP64 sums reproduces the same spread, so the gate is: at 40K rows weight
    and bias gradients rel-L2 <= 1e-3 (measured at most 8.1e-4) and the input
    gradients <= 1.5e-3 (measured 1.03e-3); at 9K rows (where one such row
    weighs more) at most 0.1% of rows off by more than 1e-2 relative and
    rel-L2 <= 1e-2.

    With zero_frac > 0 that fraction of rows gets a zero upstream gradient
    (what occluded Gaussians get): the kernel leaves them out, and their input
    gradients must come back exactly 0 although dx_items starts as NaN."""
    wl = sg.make_workload("c4", N=N, res=64, n_pairs=n_pairs)
    r = PL.renderer_for_workload(wl, precision=B.BF16)
    n = r.table.n_items
    rng = np.random.default_rng(N)
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
    dx_all = r.dx_items.double().cpu().numpy()
    assert not dx_all[:, 7:].any()            # this network has no rotation / scale inputs
    dx = dx_all[:, :7]
    rdW = [np.zeros_like(w) for w in dW]
    rdb = [np.zeros_like(b) for b in db]
    rdx = np.zeros_like(dx)
    off = 0
    for pair in wl.pairs:
        sc = wl.scenes[pair.scene]
        X = O.mlp_inputs(wl.mlp.kind, sc.mu, sc.normal, sc.vis, pair.center, pair.light)
        acts, y, Ls, Lin = O.mlp_forward(wl.mlp, X, bf16=True)
        u = up[off:off + sc.N].astype(np.float64)
        gW, gb, gX = O.mlp_backward(wl.mlp, acts, y, Ls, u[:, :3], u[:, 3], bf16=True)
        for l in range(len(gW)):
            rdW[l] += gW[l]
            rdb[l] += gb[l]
        dmu, dn, dv = O.input_grads(wl.mlp.kind, gX, sc.mu, pair.center, pair.light)
        rdx[off:off + sc.N] = np.concatenate([dmu, dn, dv[:, None]], 1)
        off += sc.N
    errs = {f"W{l}": _rel(dW[l], rdW[l]) for l in range(len(dW))}
    errs.update({f"b{l}": _rel(db[l], rdb[l]) for l in range(len(db))})
    errs["dx"] = _rel(dx, rdx)
    assert np.all(dx[zero] == 0.0) and np.isfinite(dx).all()
    row_rel = np.abs(dx - rdx).max(1) / np.maximum(np.abs(rdx).max(1), 1e-12)
    frac_bad = float((row_rel > 1e-2).mean())
    print("\nbf16 backward rel-L2 errors:", {k: f"{v:.2e}" for k, v in errs.items()},
          f"rows >1e-2: {frac_bad:.4%}")
    if int((~zero).sum()) >= 40000:
        assert all(v < (1.5e-3 if k == "dx" else 1e-3) for k, v in errs.items()), errs
    else:
        assert frac_bad <= 1e-3
        assert all(v < 1e-2 for v in errs.values()), errs


def test_bf16_pipeline_image_and_gradients():
    """Whole step with the tensor-core network (300K configuration shape,
    reduced to 20K Gaussians x 2 pairs at 96x96) vs the oracle with the
    BF16-emulating network. Raster-flagged pixels (see gpu_common) are
    excluded and get zero upstream gradient. bf16 decisions that flip between
    float32 and FP64 sums move a Gaussian's L_SSS / L_in by a few bf16 ulps,
    which reaches a pixel weighted by that Gaussian's compositing weight: the
    image gate is 99.9% of pixels within 1e-4 and all within 2e-4 (the
    measured worst pixels of the full-size batches are at 1.1-1.6e-4).
    Gradients: per tensor rel-L2 <= 1e-3, and 2e-3 for mu and v, which reach
    the network through its inputs (measured here 1.3e-3 and 1.2e-3; 3.6e-4
    and 1.3e-3 on the full-size pair). The error against the FP64 network is
    printed for the record."""
    from gpu_common import flagged, oracle_batch, run_gpu, grad_errors
    wl = sg.make_workload("c4", N=20000, res=96, n_pairs=2)
    ref0 = oracle_batch(wl, [0, 1], bf16=True)
    fl = flagged(ref0["margin"])
    dimg = sg.random_dimg(77, ref0["img"].shape[0])
    dimg[fl] = 0.0
    ref = oracle_batch(wl, [0, 1], dimg=dimg, bf16=True)
    ref64 = oracle_batch(wl, [0, 1], dimg=dimg, bf16=False)
    g = run_gpu(wl, precision=B.BF16, dimg=dimg)
    ok = ~fl
    e = np.abs(g["img"][ok] - ref["img"][ok]).max(axis=1)
    e64 = np.abs(g["img"][ok] - ref64["img"][ok]).max(axis=1)
    gerr = {k: grad_errors(g["grads"][k], ref["grads"][k])[0] for k in PL.SCENE_KEYS}
    gerr64 = {k: grad_errors(g["grads"][k], ref64["grads"][k])[0] for k in PL.SCENE_KEYS}
    werr = [grad_errors(g["dW"][l], ref["dW"][l])[0] for l in range(len(g["dW"]))]
    print(f"\nbf16 pipeline image: vs bf16 oracle max {e.max():.2e} p99.9 {np.quantile(e, 0.999):.2e}; "
          f"vs fp64 max {e64.max():.2e} mean {e64.mean():.2e}")
    print("grad rel-L2 vs bf16 oracle:", {k: f"{v:.1e}" for k, v in gerr.items()})
    print("grad rel-L2 vs fp64 oracle:", {k: f"{v:.1e}" for k, v in gerr64.items()})
    print("dW rel-L2 vs bf16 oracle:", [f"{v:.1e}" for v in werr])
    assert np.quantile(e, 0.999) <= 1e-4 and e.max() <= 2e-4
    assert all(v <= (2e-3 if k in ("mu", "vis") else 1e-3) for k, v in gerr.items()), gerr
    assert all(v <= 1e-3 for v in werr), werr
