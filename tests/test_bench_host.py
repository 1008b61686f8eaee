"""Host-side arithmetic of bench.py: the algorithmic work per point behind
every roofline fraction, the roofline and traffic bookkeeping, the fallback
peaks and the per-step launch counts.  No GPU."""
import json

import pytest

import bench
from paper_2606_29702_gb300 import workloads


def _gemm_flops(widths, C):
    """Flops of one step's jet GEMMs per point, one GEMM at a time: for every
    hidden-to-hidden layer l the forward Z = W A (M = w_l, K = w_{l-1}), the data
    gradient Abar = W^T Zbar (M = w_{l-1}, K = w_l) and the weight gradient
    Wbar = Zbar A^T (M = w_l, N = w_{l-1}, K = the C columns of the point),
    2 M N K each.  The input and output layers are not GEMMs (K = d, N = n_out)."""
    total = 0
    for l in range(2, len(widths) - 1):
        w_in, w_out = widths[l - 1], widths[l]
        total += 2 * w_out * C * w_in          # forward: M = w_out, N = C, K = w_in
        total += 2 * w_in * C * w_out          # data gradient: M = w_in, N = C, K = w_out
        total += 2 * w_out * w_in * C          # weight gradient: M = w_out, N = w_in, K = C
    return total


@pytest.mark.parametrize("name,C,expected", [
    ("burgers_2x20x4", 4, 28_800),
    ("ks_2x64x5", 6, 589_824),
    ("ns_psi_3x128x6", 13, 6_389_760),
    ("helmholtz_3x256x8", 7, 19_267_584),
])
def test_flops_per_point(name, C, expected):
    widths = workloads.WORKLOADS[name]["widths"]
    assert bench.flops_per_point(widths, C) == expected
    assert _gemm_flops(widths, C) == expected


@pytest.mark.parametrize("name,expected", [
    ("burgers_2x20x4", 1_341), ("ks_2x64x5", 16_897), ("ns_psi_3x128x6", 83_330), ("helmholtz_3x256x8", 461_825),
])
def test_parameter_counts(name, expected):
    widths = workloads.WORKLOADS[name]["widths"]
    assert workloads.n_params(widths) == expected
    assert workloads.n_params(widths) == sum(widths[i] * widths[i + 1] + widths[i + 1] for i in range(len(widths) - 1))


def test_ensemble_flops_sums_members():
    insts = [{"N": 100, "widths": [2, 32, 32, 32, 1]}, {"N": 7, "widths": [2, 128, 128, 1]}]
    assert bench.ensemble_flops(insts) == 100 * _gemm_flops([2, 32, 32, 32, 1], 4) + 7 * _gemm_flops([2, 128, 128, 1], 4)


def test_roofline_tensor_and_alu():
    peaks = {"bf16_tflops": 2000.0, "sm_max_mhz": 2000.0}
    flops = 19_267_584 * 1048576
    r = bench.roofline("bf16", flops, 40.0, peaks, "measured", traffic=123)
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s" and r["traffic"] == 123
    assert r["achieved"] == pytest.approx(flops / 0.040 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / 2000.0)
    a = bench.roofline("fp32", 1e12, 1000.0, peaks, "measured")
    assert a["bound"] == "alu" and a["peak"] == pytest.approx(152 * 128 * 2 * 2000e6 / 1e12)
    assert a["frac"] == pytest.approx(1.0 / a["peak"])
    d = bench.roofline("fp64", 1e12, 1000.0, peaks, "measured")
    assert d["peak"] == pytest.approx(152 * 2 * 2 * 2000e6 / 1e12)


def test_traffic_follows_kernel_sources(monkeypatch):
    key = ("helmholtz_3x256x8", "bf16", "store")
    assert key in bench.TRAFFIC
    nbytes, h = bench.TRAFFIC[key]
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: h)
    assert bench.traffic_for(*key) == nbytes
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)  # the kernels changed since the capture
    assert bench.traffic_for(*key) is None
    assert bench.traffic_for("no_such_workload", "bf16") is None


def test_kernel_source_hash_covers_the_sources(tmp_path, monkeypatch):
    src = tmp_path / "paper_2606_29702_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "k.cu").write_text("a")
    (src / "jet_closures_gen.h").write_text("generated")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h1 = bench.kernel_source_hash()
    (src / "jet_closures_gen.h").write_text("regenerated")  # generated from specs, not a source
    assert bench.kernel_source_hash() == h1
    (src / "k.cu").write_text("b")
    assert bench.kernel_source_hash() != h1


def test_peaks_fallback_and_measured(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    p, kind = bench.measured_peaks()
    assert kind == "fallback" and p["hbm_gbs"] == 6800.0 and p["bf16_tflops"] == 1900.0
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 7000.0, "bf16_tflops": 1850.0}))
    p, kind = bench.measured_peaks()
    assert kind == "measured" and p["bf16_tflops"] == 1850.0


def test_launches_per_step_and_schedule():
    # the headline's launch list per step: weight preparation, fused kernel,
    # weight-gradient GEMM, its partial sum, reduce + Adam
    assert bench.launches_per_step("bf16", "store") == 5
    assert bench.launches_per_step("bf16", "tile") == 3
    assert bench.launches_per_step("fp32", "tile") == 3
    assert bench.launches_per_step("bf16", "tile", dev_counter=True) == 4
    assert bench.default_schedule(workloads.WORKLOADS["helmholtz_3x256x8"], "bf16") == "store"
    assert bench.default_schedule(workloads.WORKLOADS["ns_psi_3x128x6"], "bf16") == "tile"
    assert bench.default_schedule(workloads.WORKLOADS["helmholtz_3x256x8"], "fp32") == "tile"
