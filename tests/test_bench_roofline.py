"""bench.py's roofline object, checked on the CPU from a synthetic run record:
the algorithmic work per sweep (Eq. 4's 4 N^2 flops per accepted move, the
ratio dot products and the queue append), the ceilings it is measured against,
and the rule that DRAM traffic from an ncu capture is reported only for the
source it was taken on."""
import types

import pytest

import bench


def record(N=2048, K=32, acc=0.95, steps=3, sweeps=10, ms=500.0, kinds=(2000,)):
    a = types.SimpleNamespace(steps=steps, sweeps_per_step=sweeps, gpus=1, precision="fp64",
                              workload="single", classes=[dict(N=N, K=K, batch=1)])
    nprop = sweeps * N
    res = dict(prof=[dict(sweep_kernel_ms=ms, sweep_kernels=steps * sweeps)],
               accepted=acc * nprop * steps, nprop=nprop, total_ms=ms / 0.8,
               flush_kinds=list(kinds))
    return a, res


def test_work_formula_and_emulated_ceiling():
    N, K, acc, steps, sweeps, ms = 2048, 32, 0.95, 3, 10, 500.0
    a, res = record(N, K, acc, steps, sweeps, ms)
    r = bench.roofline_for(a, res)
    props = steps * sweeps * N
    kbar = (K - 1) / 2.0
    flops = 4.0 * N * N * acc * props + 2.0 * (2 * kbar + 2) * N * props + 4.0 * kbar * N * acc * props
    assert r["achieved"] == pytest.approx(flops / (ms * 1e-3) / 1e12)
    assert r["flops_per_launch"] == pytest.approx(flops / (steps * sweeps))
    assert r["avg_launch_ms"] == pytest.approx(ms / (steps * sweeps))
    assert r["share_of_step"] == pytest.approx(0.8)
    # the emulated-fp64 flush: bound by the tensor pipe through 28 slice products
    assert r["bound"] == "tensor"
    bf16 = bench.measured_peaks().get("bf16_tflops_sustained") or 1400.0
    assert r["peak"] == pytest.approx(bf16 / 28)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["fp64_units_frac"] == pytest.approx(r["achieved"] / bench.FP64_PEAK_TFLOPS)


def test_fp64_unit_flush_is_alu_bound():
    a, res = record(kinds=(64,))
    r = bench.roofline_for(a, res)
    assert r["bound"] == "alu"
    assert r["peak"] == pytest.approx(148 * 2 * 2 * 2032e6 / 1e12)


def test_traffic_only_for_the_captured_source(monkeypatch):
    a, res = record()
    key = "%s:%s" % (bench.source_hash("kernels_sweep.cu"), "single")
    monkeypatch.setattr(bench, "NCU_TRAFFIC", {key: 1.5e8})
    assert bench.roofline_for(a, res)["traffic"] == 1.5e8
    monkeypatch.setattr(bench, "NCU_TRAFFIC", {"0123456789abcdef:single": 1.5e8})
    assert bench.roofline_for(a, res)["traffic"] is None
