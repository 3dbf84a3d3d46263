"""Host logic of bench.py on CPU: the roofline traffic field comes from an ncu
summary only while the summary's source digest matches the kernel's current
sources; a missing or stale summary gives null."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _profiles(tmp_path, monkeypatch, digest, nbytes):
    d = tmp_path / "profiles"
    d.mkdir()
    (d / "k_x_ncu.md").write_text("# summary\n\nkernel-source-sha1: %s\n\ndram-bytes-per-launch: %d\n" % (digest, nbytes))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_digest", lambda sources=None: "ab" * 20)


def test_traffic_needs_a_matching_digest(tmp_path, monkeypatch):
    _profiles(tmp_path, monkeypatch, "ab" * 20, 1234)
    assert bench.profiled_traffic("k_x") == 1234
    assert bench.profiled_traffic("k_missing") is None


def test_traffic_is_null_for_a_stale_summary(tmp_path, monkeypatch):
    _profiles(tmp_path, monkeypatch, "cd" * 20, 1234)
    assert bench.profiled_traffic("k_x") is None


def test_digest_follows_the_sources():
    a = bench.kernel_digest(bench.KERNEL_SOURCES)
    assert len(a) == 40 and a == bench.kernel_digest(bench.KERNEL_SOURCES)
    assert a != bench.kernel_digest(bench.STRIP_SOURCES)
