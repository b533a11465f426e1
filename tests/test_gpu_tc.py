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
