"""Host-side logic of bench.py: the ncu traffic figure is reported only for the trace kernel's
sources it was captured on, and the workload metadata names the benchmark configuration."""
import os
import shutil

import bench


def test_traffic_is_reported_only_for_the_captured_sources(tmp_path, monkeypatch):
    assert bench.NCU_TRAFFIC["bytes_per_launch"] > 1e9
    if bench.NCU_TRAFFIC["sources_sha256"] == bench.trace_kernel_sha256():
        assert bench.measured_traffic() == bench.NCU_TRAFFIC["bytes_per_launch"]
    else:   # the kernel changed since the capture: no figure
        assert bench.measured_traffic() is None
    # a copy with one kernel source edited no longer matches
    for rel in bench.TRACE_KERNEL_SOURCES:
        dst = tmp_path / rel
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(bench.ROOT, rel), dst)
    (tmp_path / bench.TRACE_KERNEL_SOURCES[-1]).write_text(
        (tmp_path / bench.TRACE_KERNEL_SOURCES[-1]).read_text() + "\n// edited\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_traffic() is None


def test_algorithmic_bytes_per_step():
    # 4 RK4 stages x cells per interpolation x 16 B (float4) x 2 bracketing slices
    assert bench.FIELD_BYTES_PER_STEP == 1024
    assert bench.FIELD_BYTES_BY_SCHEME == {"ngp": 128, "cic": 1024, "tsc": 3456}
