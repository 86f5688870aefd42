"""bench.py's roofline arithmetic on CPU, from made-up kernel-family
profiles: the dominant family is the one with the largest share; the bound
is the resource whose peak the family's algorithmic work needs longer on;
achieved = algorithmic work / summed launch time; frac = achieved / peak;
traffic = the stored DRAM-to-algorithmic ratio times the bytes per launch,
and only for the kernel sources the ratio was measured on."""

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

bench = pytest.importorskip("bench")
cm = pytest.importorskip("paper_2508_11608_gb300")


def _fam(ms, launches, flops, bytes_, share):
    return {"ms": ms, "launches": launches, "flops": flops, "bytes": bytes_, "share": share}


def _prof(top_bytes, top_flops):
    # family 1 (cut-patch step) dominant: 10 launches of 2 ms
    return {1: _fam(20.0, 10, top_flops, top_bytes, 0.5), 2: _fam(5.0, 10, 1e9, 1e9, 0.2),
            3: _fam(3.0, 4, 1e9, 1e9, 0.1), 4: _fam(2.0, 4, 1e8, 1e8, 0.1), 5: _fam(1.0, 8, 1e8, 1e8, 0.1)}


def test_hbm_bound_family_reports_bytes_over_time():
    hbm = 6000.0
    prof = _prof(top_bytes=60e9, top_flops=1e9)  # 60 GB in 20 ms: 3 TB/s
    r = bench._roofline(cm, prof, cm.CF_MIXED, hbm)
    assert r["kernel"] == "k_cut_warp" and r["family"] == 1
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(3000.0)
    assert r["frac"] == pytest.approx(0.5)
    assert r["per_launch_ms"] == pytest.approx(2.0)
    assert r["bytes_per_launch"] == pytest.approx(6e9)


def test_alu_bound_family_reports_flops_over_time():
    prof = _prof(top_bytes=1e6, top_flops=12.6e9)  # FP64: 12.6 GFLOP in 20 ms
    r = bench._roofline(cm, prof, cm.CF_FP64, 6000.0)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(0.63)
    assert r["frac"] == pytest.approx(0.63 / bench.FP64_PEAK_TFLOPS)


def test_traffic_needs_the_measured_sources(monkeypatch):
    prof = _prof(top_bytes=60e9, top_flops=1e9)
    key = ("k_cut_warp", "fp32")
    ratio = bench.TRAFFIC[key]["dram_over_algorithmic"]
    monkeypatch.setattr(bench, "_kernels_sha256", lambda: bench.TRAFFIC[key]["kernels_sha256"])
    r = bench._roofline(cm, prof, cm.CF_MIXED, 6000.0)
    assert r["traffic"] == pytest.approx(ratio * 6e9)
    monkeypatch.setattr(bench, "_kernels_sha256", lambda: "0" * 64)
    assert bench._roofline(cm, prof, cm.CF_MIXED, 6000.0)["traffic"] is None


def test_stored_traffic_ratios_match_the_current_kernel_sources():
    # the ratios in bench.TRAFFIC were measured on these sources; a change to
    # the kernels must come with a new capture
    for entry in bench.TRAFFIC.values():
        assert entry["kernels_sha256"] == bench._kernels_sha256()
        assert 1.0 <= entry["dram_over_algorithmic"] < 2.0
