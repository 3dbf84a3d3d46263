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


def test_binning_roofline_counts_hits_and_bins(monkeypatch):
    """Algorithmic bytes of the binning stage: per hit and per bin, with the
    bins of every layer of every event at the tuned granularity."""
    monkeypatch.setattr(bench, "measured_peaks", lambda: {"hbm_gbs": 1000.0})
    r = dict(n_events=4, L=10, n_hits=1000, tuned=dict(n_phi=8, n_w=2), stage=dict(bin=0.5))
    rl = bench.binning_roofline(r)
    bins = 4 * 10 * 8 * 2
    assert rl["bins"] == bins
    assert rl["algorithmic_bytes"] == 1000 * bench.BYTES_BIN_HIT + bins * bench.BYTES_BIN_BIN
    assert abs(rl["achieved"] - rl["algorithmic_bytes"] / 0.5e-3 / 1e9) < 1e-9
    assert abs(rl["frac"] - rl["achieved"] / 1000.0) < 1e-12
    r["stage"]["bin"] = -1.0   # stage not timed
    assert bench.binning_roofline(r)["achieved"] is None


def test_packed_buffers_hold_every_tensor_in_place():
    """The end-to-end leg moves each step's inputs, and the results it reads
    back, as one buffer each: every tensor becomes a view at a 256-byte
    aligned offset of that buffer, with its own dtype, shape and values, and
    writing through a view changes the buffer (so one copy of the buffer
    moves every tensor)."""
    import torch
    src = dict(xyz=torch.arange(30, dtype=torch.float32).reshape(3, 10),
               layer=torch.tensor([3, 1, 4, 1, 5], dtype=torch.int32),
               off=torch.tensor([0, 7, 9], dtype=torch.int64),
               empty=torch.zeros((6, 0), dtype=torch.float32))
    buf, views = bench.packed(src, "cpu")
    assert buf.dtype == torch.uint8 and buf.dim() == 1
    end = 0
    for k, v in src.items():
        w = views[k]
        assert w.dtype == v.dtype and w.shape == v.shape and torch.equal(w, v)
        if w.numel():
            off = w.data_ptr() - buf.data_ptr()
            assert off % 256 == 0 and off >= end
            end = off + w.numel() * w.element_size()
    assert end <= buf.numel()
    views["layer"][2] = 40
    copy = buf.clone()
    again = copy[views["layer"].data_ptr() - buf.data_ptr():][:20].view(torch.int32)
    assert again[2].item() == 40 and torch.equal(views["xyz"], src["xyz"])
