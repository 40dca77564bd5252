"""Host-side helpers of bench.py (CPU only): the roofline's peak and
committed-traffic lookup, and the CPU-baseline sample of each workload."""
import os

import pytest


def test_peak_is_the_measured_copy_bandwidth():
    import bench
    peak, kind = bench.measured_peaks()
    if os.path.exists(os.path.join(bench.ROOT, "MEASURED_PEAKS.json")):
        assert kind == "measured" and peak > 1000.0
    else:
        assert (peak, kind) == (6800.0, "fallback")


def test_committed_traffic_only_for_the_captured_sources(monkeypatch):
    """The traffic row counts only while the fused kernel's sources keep the
    digest it was captured on; any other digest, kernel or workload gives
    None."""
    import bench
    rows = [line for line in open(os.path.join(bench.ROOT, "profiles", "traffic.md"))
            if line.startswith("| k_fused |")]
    assert len(rows) == 1
    cells = [c.strip() for c in rows[0].strip().strip("|").split("|")]
    kernel, workload, nbytes, digest = cells
    monkeypatch.setattr(bench, "source_digest", lambda: digest)
    assert bench.committed_traffic(kernel, workload) == int(nbytes)
    assert bench.committed_traffic(kernel, "other-workload") is None
    assert bench.committed_traffic("k_other", workload) is None
    monkeypatch.setattr(bench, "source_digest", lambda: "0" * 16)
    assert bench.committed_traffic(kernel, workload) is None


def test_digest_covers_the_fused_kernel_sources():
    import bench
    d = bench.source_digest()
    assert len(d) == 16 and int(d, 16) >= 0
    for f in bench.FUSED_SOURCES:
        assert os.path.exists(os.path.join(bench.ROOT, "paper_1109_3277_gb300", "csrc", f))


def test_cpu_samples_are_bounded_sub_boxes():
    import bench
    from paper_1109_3277_gb300 import workloads as W
    w = W.spinodal(n=128)
    s, what = bench.cpu_sample_workload(w)
    assert s.shape == (96, 96, 96) and "96^3" in what
    s1, what1 = bench.cpu_sample_workload("spinodal", 64)
    assert s1.shape == (64, 64, 64) and "64^3" in what1
    a = W.adsorption_box()
    s2, what2 = bench.cpu_sample_workload(a)
    assert s2 is a and what2 == "the full workload"
