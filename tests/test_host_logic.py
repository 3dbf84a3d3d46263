"""Host logic of the package on CPU: the binding's argument checks (before
any library call) and the autotuner's launch choices and on-disk cache."""
import os
import sys

import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2002_06295_gb300 import api, tune  # noqa: E402


def test_pointer_marshalling_checks_device_dtype_and_layout():
    """Only contiguous CUDA tensors of the declared dtype reach the library;
    None passes as a null pointer."""
    assert api._ptr(None) is None
    with pytest.raises(TypeError, match="CUDA tensor"):
        api._ptr(torch.zeros(4), torch.float32, "xyz")
    with pytest.raises(TypeError, match="CUDA tensor"):
        api._ptr([1.0, 2.0], torch.float32, "xyz")


def test_lane_choices_are_powers_of_two_from_the_candidate_count():
    """Lanes per seed: powers of two from the first one holding max_cands
    candidates (one lane each) up to a warp."""
    assert tune.lane_choices(1) == [1, 2, 4, 8, 16, 32]
    assert tune.lane_choices(4) == [4, 8, 16, 32]
    assert tune.lane_choices(6) == [8, 16, 32]
    assert tune.lane_choices(8) == [8, 16, 32]
    assert tune.lane_choices(32) == [32]


def test_autotune_cache_round_trip(tmp_path, monkeypatch):
    """The cache file is written atomically and read back; a missing or
    corrupt file reads as empty, and an unwritable place is ignored."""
    monkeypatch.setenv("MKF_CACHE_DIR", str(tmp_path / "c"))
    assert tune._load_cache() == {}
    entry = {"k|1": dict(n_phi=64, n_w=16, warps=8, lanes=8, ms=0.8)}
    tune._store_cache(entry)
    assert tune._load_cache() == entry
    assert not [f for f in os.listdir(tmp_path / "c") if ".tmp" in f]
    (tmp_path / "c" / "autotune.json").write_text("{not json")
    assert tune._load_cache() == {}
    blocker = tmp_path / "file"
    blocker.write_text("x")
    monkeypatch.setenv("MKF_CACHE_DIR", str(blocker / "sub"))
    tune._store_cache(entry)   # cannot create a directory under a file: ignored
    assert tune._load_cache() == {}


def test_bin_choices_fit_the_binning_limits():
    """Every (phi bins, w bins) the autotuner tries is accepted by
    mkf_load_geometry (1..4096 of each per layer), and on every workload the
    finest choice keeps the bin keys (event, layer, bin) within int32."""
    import synth
    assert len(set(tune.BIN_CHOICES)) == len(tune.BIN_CHOICES)
    for n_phi, n_w in tune.BIN_CHOICES:
        assert 1 <= n_phi <= 4096 and 1 <= n_w <= 4096
    assert all(w in (2, 4, 8) for w in tune.WARP_CHOICES)
    finest = max(p * w for p, w in tune.BIN_CHOICES)
    for cid, spec in synth.WORKLOAD_SPECS.items():
        n_keys = spec["n_events"] * spec["geom"]().n_layers * finest
        assert n_keys < 2 ** 31, (cid, n_keys)
