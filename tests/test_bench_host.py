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
    monkeypatch.setattr(bench, "render_source_sha", lambda: "0" * 64)
    assert bench.kernel_traffic("render_bwd", "c4", 64) is None      # source changed since the capture


def test_alu_work_reproduces_the_reported_figure():
    """The 64-pair step's counters (2.92G contributions, 9.03G alpha
    evaluations, 41M pixels) over 27.56 ms give 14.7 TFLOP/s."""
    c, e, px = 2924266653, 9026382678, 64 * 800 * 800
    fl = bench.FLOP_BWD_CONTRIB * c + bench.FLOP_EVAL * (e - c) + bench.FLOP_SHADE_BWD * px
    assert abs(fl / 27.56e-3 / 1e12 - 14.69) < 0.01
    assert abs(bench.ALU_PEAK_TFLOPS - 80.548) < 1e-3


def test_mlp_flops_counts_two_per_multiply_add():
    assert bench.mlp_flops([64, 128, 128, 128, 128, 4], 1) == 2 * (64 * 128 + 3 * 128 * 128 + 128 * 4)
    assert bench.mlp_flops([9, 32, 4], 10) == 10 * 2 * (9 * 32 + 32 * 4)
