"""Host logic of bench.py (no GPU): the DRAM traffic figure is reported only
for the kernel source it was measured on and for workloads made of the
captured pair shape; the per-unit work constants give the documented
achieved figure; the network FLOP count matches the layer widths."""
import bench


def test_traffic_only_for_the_measured_source_and_workload(monkeypatch):
    sha, per_pair = bench.KERNEL_TRAFFIC["render_bwd"]
    assert len(bench.render_source_sha()) == 64
    monkeypatch.setattr(bench, "render_source_sha", lambda: sha)    # as if the source were the captured one
    assert bench.kernel_traffic("render_bwd", "c4", 64) == per_pair * 64
    assert bench.kernel_traffic("render_bwd", "c5", 64) is None     # other pair shapes
    assert bench.kernel_traffic("mlp_bwd", "c4", 64) is None         # no capture for that stage
    assert bench.kernel_traffic("render_bwd", "c4", 64, (8, 32)) is None    # another schedule
    assert bench.kernel_traffic("render_bwd", "c4", 64, (16, 64)) is None
    monkeypatch.setattr(bench, "render_source_sha", lambda: "0" * 64)
    assert bench.kernel_traffic("render_bwd", "c4", 64) is None      # source changed since the capture


def test_alu_work_reproduces_the_reported_figure():
    """The 64-pair step's counters (2.92G contributions, 9.03G alpha
    evaluations, 41M pixels) over 26.35 ms give 15.0 TFLOP/s."""
    c, e, px = 2924266653, 9026382678, 64 * 800 * 800
    fl = bench.FLOP_BWD_CONTRIB * c + bench.FLOP_EVAL * (e - c) + bench.FLOP_SHADE_BWD * px
    assert abs(fl / 26.35e-3 / 1e12 - 15.03) < 0.01
    assert abs(bench.ALU_PEAK_TFLOPS - 80.548) < 1e-3


def test_mlp_flops_counts_two_per_multiply_add():
    assert bench.mlp_flops([64, 128, 128, 128, 128, 4], 1) == 2 * (64 * 128 + 3 * 128 * 128 + 128 * 4)
    assert bench.mlp_flops([9, 32, 4], 10) == 10 * 2 * (9 * 32 + 32 * 4)


def test_parity_report_gates_unflagged_pixels(monkeypatch):
    """The bench's parity object: pixels whose oracle decision margin is below
    the flag margin are counted, not gated; the max error of the others is
    compared with the gate."""
    import numpy as np
    pix = {0: np.zeros((4, 2), np.int32), 5: np.zeros((3, 2), np.int32)}
    got = {0: np.full((4, 3), 0.5), 5: np.full((3, 3), 0.25)}
    ref = {"img_0": np.full((4, 3), 0.5 + 5e-5), "margin_0": np.array([[1.0, 1.0, 0]] * 3 + [[1e-6, 1.0, 0]]),
           "img_5": np.full((3, 3), 0.25), "margin_5": np.ones((3, 3)),
           "img64_0": np.full((4, 3), 0.5 + 2e-3), "img64_5": np.full((3, 3), 0.25)}
    ref["img_0"][3] = 0.9                      # a flagged pixel with a large error is left out of the gate
    monkeypatch.setattr(bench, "cpu_oracle_pixels", lambda *a, **k: (ref, 1.5))

    class A:
        workload, net, pairs = "c4", None, None
    out = bench.parity_report(A, 64, pix, got, True)
    assert out["pixels"] == 7 and out["flagged"] == 1
    assert abs(out["max_err"] - 5e-5) < 1e-12 and out["pass"] and out["failing"] == 0
    assert abs(out["vs_fp64_network"]["max_err"] - 2e-3) < 1e-12
