"""bench.py's host logic on the CPU: the roofline position of the dominant kernel (which kernel, which bound,
achieved over peak, share, per-launch figures) and when the captured DRAM traffic may be reported beside it
(only while the kernel runs the launch variant the capture measured), and the read-back of the autotuner's
choices through the library's host-only cache writer."""

import json

import pytest

import bench
import paper_1912_10082_gb300 as st

HBM = 6690.8


def test_roofline_hbm_bound_dominant_kernel():
    prof = {"ts_tn_df": dict(launches=10, ms=20.0, bytes=8.0e10, flops=1.0e10),
            "fd_gemm32": dict(launches=100, ms=5.0, bytes=1.0e9, flops=1.0e10)}
    r = bench.roofline_of(prof, HBM)
    assert r["kernel"] == "ts_tn_df" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(8.0e10 / 0.020 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / HBM)
    assert r["share"] == pytest.approx(20.0 / 25.0)
    assert r["ms_per_launch"] == pytest.approx(2.0) and r["bytes_per_launch"] == pytest.approx(8.0e9)
    assert r["traffic"] is None   # no capture for this kernel


def test_roofline_fp64_alu_bound_and_traffic_by_variant():
    prof = {"fd_gemm64": dict(launches=160, ms=4.3, bytes=2.1e8, flops=2.65e9),
            "ts_tn": dict(launches=260, ms=3.0, bytes=1e9, flops=1e8)}
    r = bench.roofline_of(prof, HBM)
    assert r["bound"] == "alu" and r["alu"] == "fp64" and r["peak"] == bench.FP64_PEAK_TFLOPS
    assert r["achieved"] == pytest.approx(2.65e9 / 4.3e-3 / 1e12)
    tr = json.loads((bench.ROOT / "profiles" / "traffic.json").read_text())["fd_gemm64"]
    assert r["traffic"] == tr["bytes_per_launch"]          # built-in choices: the captured variant
    same = {"fd_gemm64": {tr["variant"]: 3}}
    assert bench.roofline_of(prof, HBM, same)["traffic"] == tr["bytes_per_launch"]
    other = {"fd_gemm64": {tr["variant"]: 2, "tile64": 1}}
    assert bench.roofline_of(prof, HBM, other)["traffic"] is None
    assert bench.roofline_of(prof, HBM, {"fd_gemm32": {"tile64": 1}})["traffic"] == tr["bytes_per_launch"]
    assert bench.roofline_of({}, HBM) is None


def test_choice_summary_names_variants():
    rows = [(1, 8, 0, 255, 255, 1, 0), (1, 8, 1, 255, 255, 1, 0), (1, 4, 0, 255, 255, 2, 2),
            (2, 8, 255, 510, 2, 0, 1), (2, 4, 63, 7938, 3, 0, 0)]
    assert bench.choice_summary(rows) == {"fd_gemm64": {"tile16": 2}, "fd_gemm32": {"tile64": 1},
                                          "line64": {"thread_64_steps": 1}, "line32": {"warp_per_row": 1}}
    assert bench.choice_summary(None) is None and bench.choice_summary([]) == {}


def test_tuned_choices_read_back_through_the_library(tmp_path):
    from paper_1912_10082_gb300.build import build

    build()
    L = st.lib()
    L.st_autotune_reset()
    try:
        src = tmp_path / "c.txt"
        src.write_text("st-autotune 1\ndevice bench\n1 8 1 255 255 2 2\n2 4 63 7938 3 0 1\n")
        assert st.autotune_load(src, "bench") == 2
        rows = bench.tuned_choices(st)
        assert sorted(rows) == [(1, 8, 1, 255, 255, 2, 2), (2, 4, 63, 7938, 3, 0, 1)]
        assert bench.choice_summary(rows) == {"fd_gemm64": {"tile64": 1}, "line32": {"thread_64_steps": 1}}
    finally:
        L.st_autotune_reset()
    assert bench.tuned_choices(st) == []
