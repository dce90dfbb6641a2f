"""bench.py's roofline arithmetic on the CPU, against figures worked out by
hand for the bench workload (2D heat 128^2, N = 512 slices, m = 50 RK4 steps,
batch 8) and the GB300's 152 SMs at 2070 MHz:

* point-steps per fine launch: 8 x 512 x 50 x 16384 = 3,355,443,200;
* FP32 pipe: 128 lanes/clk/SM x 152 x 2.07e9 = 40.27392 T lane-ops/s;
* the method's work: 20 FP32 lane-ops per point-step (the Horner RK4,
  4 stages x (3 FADD + 2 FFMA)), whatever arithmetic carries it out, so a
  21.889 ms float-float launch runs 3.3554e9 x 20 / 21.889e-3 = 3.0658 T
  method lane-ops/s = 7.61% of the pipe (frac); it executes 179 lane-ops per
  point-step, 27.439 T lane-ops/s = 68.1% (frac_executed);
* the split RK4 kernel executes 69 lane-ops per point-step;
* algorithmic bytes per launch: x read once in FP64 (x_{n-1} and x_n are
  the same array), the row written in FP64 (residuals) or FP32 (inner
  solves): 16 or 12 bytes per point-slice of 8 x 512 x 16384.
"""
import math

import pytest

import bench
from paper_2203_10148_gb300 import inputs

PEAKS = {"sm_max_mhz": 2070.0, "bf16_tflops": 1925.6}
EMPTY = {"fine_fp32": (0, 0.0), "fine_fp64": (0, 0.0), "fine_ff": (0, 0.0), "fine_split": (0, 0.0)}


def _bench_workload():
    return bench.workload(bench.parse([]), 0)


def test_bench_workload_shape():
    w = _bench_workload()
    assert (w.kind, w.batch, w.N, w.M, w.fine[1]) == ("heat2d", 8, 512, 128 * 128, 50)


def test_float_float_fine_kernel_roofline():
    w = _bench_workload()
    timing = dict(EMPTY, fine_ff=(10, 218.89436721801758), fine_fp32=(30, 83.55587142705917))
    r = bench.roofline(w, timing, PEAKS, 152)
    assert r["bound"] == "alu" and r["kernel"] == "k_heat2d_fine<ff>"
    assert math.isclose(r["peak"], 40.27392, rel_tol=1e-12)
    assert math.isclose(r["launch_ms"], 21.889436721801758, rel_tol=1e-12)
    assert math.isclose(r["achieved"], 3355443200 * 20 / 21.889436721801758e-3 / 1e12, rel_tol=1e-12)
    assert r["achieved"] == pytest.approx(3.0658, abs=5e-4)
    assert r["frac"] == pytest.approx(0.07612, abs=5e-5)
    assert r["frac_executed"] == pytest.approx(0.6813, abs=5e-5)
    assert r["algorithmic_bytes"] == 8 * 512 * 16384 * 16
    # the FP32 kernel of the same solves: 20 lane-ops per point-step
    assert r["fine_fp32"]["achieved"] == pytest.approx(3355443200 * 20 / (83.55587142705917 / 30 * 1e-3) / 1e12,
                                                       rel=1e-12)


def test_fp32_dominant_and_no_fine_work():
    w = _bench_workload()
    r = bench.roofline(w, dict(EMPTY, fine_fp32=(4, 12.0)), PEAKS, 152)
    assert r["kernel"] == "k_heat2d_fine<float>"
    assert r["achieved"] == pytest.approx(3355443200 * 20 / 3.0e-3 / 1e12, rel=1e-12)
    assert r["algorithmic_bytes"] == 8 * 512 * 16384 * 12
    assert r["frac"] == r["frac_executed"]
    assert bench.roofline(w, EMPTY, PEAKS, 152) is None


def test_split_fine_kernel_roofline():
    w = _bench_workload()
    r = bench.roofline(w, dict(EMPTY, fine_split=(2, 17.0), fine_fp32=(6, 10.0)), PEAKS, 152)
    assert r["kernel"] == "k_heat2d_split"
    assert r["frac"] == pytest.approx(3355443200 * 20 / 8.5e-3 / 1e12 / 40.27392, rel=1e-12)
    assert r["frac_executed"] == pytest.approx(3355443200 * 69 / 8.5e-3 / 1e12 / 40.27392, rel=1e-12)
    assert r["algorithmic_bytes"] == 8 * 512 * 16384 * 16


def test_dense_tensor_roofline_takes_half_the_bf16_peak():
    w = inputs.dense(M=1024, N=4096, T=10.0, fine_steps=200)
    r = bench.roofline(w, dict(EMPTY, fine_fp32=(2, 0.228)), PEAKS, 152)
    assert r["bound"] == "tensor" and math.isclose(r["peak"], 1925.6 / 2, rel_tol=1e-12)
    # three TF32 products of 2 M^2 N flop each, per 0.114 ms launch
    assert r["achieved"] == pytest.approx(3 * 2 * 1024 * 1024 * 4096 / 0.114e-3 / 1e12, rel=1e-12)
