"""The bench's `traffic` figure comes from a committed ncu summary and is reported only while
the kernel's sources are the ones the counters were taken on.  CPU only."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_every_profiled_kernel_has_a_summary_with_hash_and_bytes():
    for kernel, path in bench.PROFILE_SUMMARY.items():
        text = open(os.path.join(ROOT, path)).read()
        assert "source_sha256" in text, kernel
        assert kernel in bench.KERNEL_SOURCES
        for f in bench.KERNEL_SOURCES[kernel]:
            assert os.path.exists(os.path.join(ROOT, "paper_1609_01317_gb300", "csrc", f))


def test_traffic_is_withheld_when_the_sources_changed(monkeypatch):
    # a summary whose recorded hash matches gives its bytes; any other hash gives None
    for kernel in ("k_march", "k_adjoint"):
        text = open(os.path.join(ROOT, bench.PROFILE_SUMMARY[kernel])).read()
        recorded = text.split("source_sha256:")[1].split("`")[1]
        monkeypatch.setattr(bench, "source_hash", lambda k, r=recorded: r)
        got = bench.profiled_traffic(kernel)
        assert got is not None and got > 1e6
        monkeypatch.setattr(bench, "source_hash", lambda k: "0" * 64)
        assert bench.profiled_traffic(kernel) is None


def test_source_hash_covers_the_launch_descriptors():
    for kernel in ("k_march", "k_adjoint", "k_surface"):
        assert "vr_internal.h" in bench.KERNEL_SOURCES[kernel]
        assert len(bench.source_hash(kernel)) == 64
