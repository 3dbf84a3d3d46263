"""Allocation-free duplicate removal (mkf_dedup_tracks_noalloc) through the C
ABI.  It serves callers that cannot allocate device memory while running; its
working memory is one fixed array in the library.  Its flags must equal those
of the context-based mkf_dedup_tracks on the same tracks, on two calls in a row
(the fixed array keeps the previous call's contents, so the second call checks
that everything that must start fresh is reset).

This file is collected last on purpose."""
import numpy as np
import pytest
import torch

import synth
from _util import f32, i32, i64, make_ctx, oracle_build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _track_lists():
    """Two inputs: the oracle's C1 tracks, and a synthetic list of two events
    with heavy overlaps and exact score ties."""
    ev = synth.make_config_event(1)
    ref = oracle_build([ev], max_cands=4)
    a = (ref["hits"], ref["score"].astype(np.float32), ref["nhits"], np.array([0, ev.n_seeds]), ev.n_hits)
    rng = np.random.default_rng(9)
    S, L, Hn = 3000, 10, 4000
    hits = np.full((S, L), -1, np.int32)
    nh = rng.integers(2, L + 1, S).astype(np.int32)
    for s in range(S):
        hits[s, :nh[s]] = rng.choice(Hn, nh[s], replace=False) if rng.random() < 0.5 else \
            (rng.integers(0, 40) * 100 + rng.choice(60, nh[s], replace=False))
    hits[1000:] = np.where(hits[1000:] >= 0, hits[1000:] + Hn, -1)
    score = np.round(rng.normal(30, 10, S), 1).astype(np.float32)
    b = (hits, score, nh, np.array([0, 1000, S]), 2 * Hn)
    return ev.geom, [a, b]


def test_noalloc_matches_context_dedup_twice_in_a_row():
    import paper_2002_06295_gb300 as mkf
    dev = torch.device("cuda", 0)
    geom, inputs = _track_lists()
    ctx = make_ctx(geom)
    for hits, score, nh, soff, H in inputs:
        hd, sd, nd, od = i32(hits, dev), f32(score, dev), i32(nh, dev), i64(soff, dev)
        ref = mkf.mkf_dedup_tracks(ctx, hd, sd, nd, od, H)
        mkf.mkf_sync(ctx)
        for _ in range(2):
            flags = torch.full((hits.shape[0],), -7, dtype=torch.int32, device=dev)
            status = torch.full((1,), -1, dtype=torch.int32, device=dev)
            rc = mkf.mkf_dedup_tracks_noalloc(hd, sd, nd, od, H, out_flags=flags, out_status=status)
            torch.cuda.synchronize()
            assert rc == 0
            assert int(status.item()) == 0
            assert torch.equal(flags, ref)
    ctx.close()


def test_noalloc_calls_allocate_no_device_memory():
    """The property the entry point exists for: once the outputs exist, further
    calls leave the device's free memory unchanged (no cudaMalloc inside)."""
    import paper_2002_06295_gb300 as mkf
    dev = torch.device("cuda", 0)
    _, inputs = _track_lists()
    hits, score, nh, soff, H = inputs[1]
    hd, sd, nd, od = i32(hits, dev), f32(score, dev), i32(nh, dev), i64(soff, dev)
    flags = torch.empty(hits.shape[0], dtype=torch.int32, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    assert mkf.mkf_dedup_tracks_noalloc(hd, sd, nd, od, H, out_flags=flags, out_status=status) == 0
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(dev)[0]
    for _ in range(5):
        assert mkf.mkf_dedup_tracks_noalloc(hd, sd, nd, od, H, out_flags=flags, out_status=status) == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info(dev)[0] == free0
    assert int(status.item()) == 0


def test_event_offsets_past_the_tracks_are_clamped():
    """An over-long last event offset (S + 5 for S tracks) must not make either
    entry point read or write past the track arrays: both flag it as bad input
    and still give the flags of the correct offsets for the S tracks."""
    import paper_2002_06295_gb300 as mkf
    dev = torch.device("cuda", 0)
    geom, inputs = _track_lists()
    hits, score, nh, soff, H = inputs[1]
    S = hits.shape[0]
    hd, sd, nd = i32(hits, dev), f32(score, dev), i32(nh, dev)
    ctx = make_ctx(geom)
    ref = mkf.mkf_dedup_tracks(ctx, hd, sd, nd, i64(soff, dev), H)
    mkf.mkf_sync(ctx)
    bad_off = np.array(soff, np.int64)
    bad_off[-1] = S + 5
    flags_ctx = mkf.mkf_dedup_tracks(ctx, hd, sd, nd, i64(bad_off, dev), H)
    with pytest.raises(mkf.MkfError) as err:
        mkf.mkf_sync(ctx)
    assert err.value.code == -1   # MKF_ERR_ARG: an input index out of range
    assert torch.equal(flags_ctx, ref)
    flags = torch.full((S,), -7, dtype=torch.int32, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    rc = mkf.mkf_dedup_tracks_noalloc(hd, sd, nd, i64(bad_off, dev), H, out_flags=flags, out_status=status)
    torch.cuda.synchronize()
    assert rc == 0
    assert int(status.item()) & 4
    assert torch.equal(flags, ref)
    # the next call with correct offsets starts clean
    rc = mkf.mkf_dedup_tracks_noalloc(hd, sd, nd, i64(soff, dev), H, out_flags=flags, out_status=status)
    torch.cuda.synchronize()
    assert rc == 0 and int(status.item()) == 0 and torch.equal(flags, ref)
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_array():
    import paper_2002_06295_gb300 as mkf
    dev = torch.device("cuda", 0)
    S = 16385
    hits = torch.full((S, 4), -1, dtype=torch.int32, device=dev)
    flags = torch.empty(S, dtype=torch.int32, device=dev)
    rc = mkf.mkf_dedup_tracks_noalloc(hits, torch.zeros(S, device=dev), torch.zeros(S, dtype=torch.int32, device=dev),
                                      i64([0, S], dev), 100, out_flags=flags)
    assert rc == -6   # MKF_ERR_CAPACITY
    rc = mkf.mkf_dedup_tracks_noalloc(hits[:10], torch.zeros(10, device=dev),
                                      torch.zeros(10, dtype=torch.int32, device=dev), i64([0, 10], dev), 524289,
                                      out_flags=flags[:10])
    assert rc == -6
