"""Host logic of bench.py (no GPU): the roofline arithmetic of both schedules
on synthetic per-kind totals, the parity check's per-sample slicing and
tolerance, and the rule that a DRAM traffic record counts only for the kernel
sources and plan it was captured on."""
import json

import numpy as np
import pytest

import bench

PEAKS = {"hbm_gbs": 6000.0, "bf16_tflops": 2000.0, "bf16_tflops_sustained": 1500.0, "sm_max_mhz": 2000.0}


def test_tensor_roofline_is_bytes_per_launch_over_launch_time():
    by_kind = {"block_bwd": dict(launches=26, ms=52.0, flops=26 * 4e12 * 2e-3, bytes=26 * 6000e9 * 2e-3),
               "block_fwd": dict(launches=26, ms=26.0, flops=0.0, bytes=26 * 3000e9 * 1e-3),
               "post": dict(launches=3, ms=2.0, flops=0.0, bytes=1e9)}
    info = {"window": 5, "passes": 26, "variant": 0}
    roof, hbm = bench.tensor_roofline(by_kind, info, 80.0, PEAKS, "measured")
    # 12 GB per launch in 2 ms: 6000 GB/s, the whole peak
    assert roof["bound"] == "hbm" and roof["unit"] == "GB/s"
    assert roof["achieved"] == pytest.approx(6000.0) and roof["frac"] == pytest.approx(1.0)
    assert roof["ms_per_launch"] == pytest.approx(2.0) and roof["share_of_step"] == pytest.approx(52.0 / 80.0)
    # 8 GFLOP per launch in 2 ms: 4 TFLOP/s of the 1500 sustained
    assert roof["tensor_pipe"]["achieved_tflops"] == pytest.approx(4.0)
    assert roof["tensor_pipe"]["frac"] == pytest.approx(4.0 / 1500.0)
    assert roof["forward_kernel"]["achieved"] == pytest.approx(3000.0)
    # block passes only: 26 x (12 + 3) GB over 78 ms
    assert hbm["achieved_gbs"] == pytest.approx((26 * 12e9 + 26 * 3e9) / 78e-3 / 1e9)
    assert hbm["frac"] == pytest.approx(hbm["achieved_gbs"] / 6000.0)


def test_window_roofline_counts_backward_and_turnaround_kernels():
    by_kind = {"pass_bwd": dict(launches=3, ms=30.0, flops=3 * 1e12 * 10e-3, bytes=3 * 5e9 * 10e-3),
               "pass_turnaround": dict(launches=1, ms=10.0, flops=1e12 * 10e-3, bytes=5e9 * 10e-3),
               "pass_fwd": dict(launches=3, ms=15.0, flops=3 * 2e12 * 5e-3, bytes=0.0),
               "prep": dict(launches=1, ms=1.0, flops=0.0, bytes=0.0)}
    info = {"window": 12, "threads": 256, "variant": 2, "passes": 4, "checkpoint_stride": 1}
    roof, hbm = bench.window_roofline(by_kind, info, 56.0, PEAKS, "measured")
    alu = 152 * 128 * 2 * 2000.0e6 / 1e12
    assert roof["bound"] == "alu" and roof["peak"] == pytest.approx(alu)
    assert roof["achieved"] == pytest.approx(1.0) and roof["launches_per_step"] == 4
    assert roof["hbm"]["achieved_gbs"] == pytest.approx(5.0)
    assert "packed" in roof["kernel"]
    assert hbm["bytes_per_step"] == pytest.approx(4 * 5e9 * 10e-3)


def test_parity_check_slices_per_sample_outputs_and_applies_the_tolerance():
    rng = np.random.default_rng(0)
    o = {"T": rng.normal(size=4) + 1j, "Omega": rng.normal(size=4) + 0j, "grad": rng.normal(size=8),
         "hvp": rng.normal(size=8), "E": rng.normal(size=(4, 3)), "DE": rng.normal(size=(4, 3))}
    d = {"T": np.concatenate([o["T"], [9.0]]), "Omega": np.concatenate([o["Omega"], [9.0]]),
         "grad": o["grad"] * (1 + 1e-7), "hvp": o["hvp"].copy()}
    r = bench.parity_check(d, o, 4)
    assert r["pass"] and set(k for k in r if k.endswith("_rel")) == {"T_rel", "Omega_rel", "grad_rel", "hvp_rel"}
    d["hvp"] = o["hvp"] + 1e-3 * np.linalg.norm(o["hvp"])
    assert not bench.parity_check(d, o, 4)["pass"]
    w = {"T": o["T"], "Omega": o["Omega"], "E": o["E"], "DE": o["DE"] * 1.01}
    r = bench.parity_check(w, o, 4)
    assert set(k for k in r if k.endswith("_rel")) == {"T_rel", "Omega_rel", "E_rel", "DE_rel"}
    assert not r["pass"] and r["DE_rel"] == pytest.approx(0.01)


def test_traffic_record_needs_matching_sources_and_plan(tmp_path, monkeypatch):
    f = tmp_path / "traffic.json"
    monkeypatch.setitem(bench.TRAFFIC_FILES, "tensor", str(f))
    info = {"window": 5, "passes": 26, "variant": 0}
    rec = {"plan": dict(info), "bwd_kernel_bytes_per_launch": 3.5e9}
    f.write_text(json.dumps({"source_sha256": bench.kernel_source_hash("tensor"), "records": [rec]}))
    assert bench.recorded_traffic(info, "tensor") == 3.5e9
    assert bench.recorded_traffic(dict(info, passes=25), "tensor") is None
    f.write_text(json.dumps({"source_sha256": "0" * 64, "records": [rec]}))
    assert bench.recorded_traffic(info, "tensor") is None
    assert bench.kernel_source_hash("tensor") != bench.kernel_source_hash("window")
