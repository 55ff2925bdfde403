"""Host-side logic of bench.py: the ncu record (DRAM traffic, instructions per RK4 step) is reported
only for the trace kernel code it was captured on, comments do not count as code, the roofline
arithmetic, and the workload metadata names the benchmark configuration."""
import os
import shutil

import bench


def _copy_sources(tmp_path):
    for rel in bench.TRACE_KERNEL_SOURCES:
        dst = tmp_path / rel
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(bench.ROOT, rel), dst)


def test_ncu_record_is_reported_only_for_the_captured_code(tmp_path, monkeypatch):
    if bench.NCU_RECORD["sources_sha256"] == bench.trace_kernel_sha256():
        assert bench.ncu_record() is bench.NCU_RECORD
        assert bench.measured_traffic() == bench.NCU_RECORD["dram_bytes_per_launch"]
    else:   # the kernel changed since the capture: no figure
        assert bench.ncu_record() is None and bench.measured_traffic() is None
    _copy_sources(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    base = bench.trace_kernel_sha256()
    last = tmp_path / bench.TRACE_KERNEL_SOURCES[-1]
    # a comment changes nothing
    last.write_text(last.read_text() + "\n// a remark\n/* and a block\n   comment */\n")
    assert bench.trace_kernel_sha256() == base
    # code does
    last.write_text(last.read_text() + "\nstatic int edited = 1;\n")
    assert bench.trace_kernel_sha256() != base
    monkeypatch.setattr(bench, "NCU_RECORD", dict(bench.NCU_RECORD, sources_sha256=base))
    assert bench.ncu_record() is None


def test_comment_stripping_keeps_strings():
    src = 'int a; // x\n/* y */ const char* s = "//kept"; char c = \'/\';'
    out = bench._strip_comments(src)
    assert "//kept" in out and "x" not in out.replace("//kept", "") and "'/'" in out


def test_roofline_arithmetic():
    rec = {"sources_sha256": "x", "dram_bytes_per_launch": 50e9,
           "per_rk4_step": {"warp_inst": 100.0, "fp64_lane_slots": 64.0}, "pct": {}}
    r = bench.roofline(1e9, 500.0, 2000.0, 5e11, 6700.0, 1024, rec, "test")
    steps_per_s = 1e9 / 0.5
    assert r["bound"] == "alu"
    assert abs(r["achieved"] - 64.0 * steps_per_s / 1e9) < 1e-9
    assert abs(r["frac"] - 64.0 * steps_per_s / 5e11) < 1e-12
    assert abs(r["issue"]["frac"] - 100.0 * steps_per_s / (152 * 4 * 2000e6)) < 1e-12
    assert abs(r["dram"]["achieved_GBs"] - 100.0) < 1e-9 and r["traffic"] == 50e9
    assert abs(r["hbm_effective"]["achieved_GBs"] - 1024 * steps_per_s / 1e9) < 1e-6
    stale = bench.roofline(1e9, 500.0, 2000.0, 5e11, 6700.0, 1024, None, "test")
    assert stale["achieved"] is None and stale["traffic"] is None
    assert stale["ncu_record"].startswith("stale")
    other = bench.roofline(1e9, 500.0, 2000.0, 5e11, 6700.0, 1024, None, "test", "covers another workload")
    assert other["ncu_record"] == "covers another workload" and other["frac"] is None


def test_algorithmic_bytes_per_step():
    # 4 RK4 stages x cells per interpolation x 16 B (float4) x 2 bracketing slices
    assert bench.FIELD_BYTES_PER_STEP == 1024
    assert bench.FIELD_BYTES_BY_SCHEME == {"ngp": 128, "cic": 1024, "tsc": 3456}
