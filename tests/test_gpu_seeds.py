"""Hit-based seeding on the GPU (four innermost barrel layers, Sec. 3) against
the FP64 oracle.  Decisions are FP32 on the GPU and FP64 in the oracle, so
quadruplets within EPS (relative) of a cut may go either way: every GPU seed
must be one the oracle passes with margin >= -EPS, and every oracle seed with
margin >= EPS must be found.  The parameters of common seeds agree within
tolerances derived from FP32 hit records (positions to ~1e-6 cm): z0 1e-4 cm,
kappa 2e-4 /GeV + 2e-4 relative, phi and theta 2e-5 rad.  Also: event offsets,
masked hits, the capacity report, and tracks built from hit seeds."""
import numpy as np
import pytest
import torch

import synth.events as sev

pytestmark = pytest.mark.gpu

EPS = 1e-3
CUTS = dict(pt_min=0.5, z_max=5.0, rphi_tol=0.05, z_tol=0.1)
CUTS_B10 = dict(pt_min=0.5, z_max=5.0, rphi_tol=0.15, z_tol=0.3)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _ctx_for(batch):
    from tests._util import make_ctx
    return make_ctx(batch.geom)


def _bin(ctx, xyz, lcov, layer, off, mask=None):
    import paper_2002_06295_gb300 as mkf
    dev = torch.device("cuda", 0)
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(dev, dt)
    args = (t(xyz.T, torch.float32), t(lcov.T, torch.float32), t(layer, torch.int32), t(off, torch.int64))
    if mask is None:
        mkf.mkf_bin_hits(ctx, *args)
    else:
        mkf.mkf_bin_hits_masked(ctx, *args, mask=t(mask, torch.uint8))


def _compare(got, ref_loose, ref, off):
    n = got["n"]
    gh = got["hits"].cpu().numpy()
    gset = {tuple(h): i for i, h in enumerate(gh)}
    assert len(gset) == n, "duplicate seeds"
    loose = {tuple(h): i for i, h in enumerate(ref_loose["hits"])}
    strong = {tuple(h) for h, m in zip(ref["hits"], ref["margin"]) if m >= EPS}
    missing = strong - gset.keys()
    extra = gset.keys() - loose.keys()
    assert not missing, "%d oracle seeds not found, e.g. %s" % (len(missing), sorted(missing)[:3])
    assert not extra, "%d GPU seeds outside the oracle's cut band, e.g. %s" % (len(extra), sorted(extra)[:3])
    # parameters
    gp = got["par"].cpu().numpy()
    for q, i in gset.items():
        j = loose[q]
        p, r = gp[:, i], ref_loose["par"][j]
        assert abs(p[2] - r[2]) < 1e-4, (q, p, r)
        assert abs(p[3] - r[3]) < 2e-4 + 2e-4 * abs(r[3]), (q, p, r)
        assert abs(np.remainder(p[4] - r[4] + np.pi, 2 * np.pi) - np.pi) < 2e-5, (q, p, r)
        assert abs(p[5] - r[5]) < 2e-5, (q, p, r)
        assert p[0] == 0.0 and p[1] == 0.0
    # event offsets: seeds of event e use hits of event e only
    eo = got["ev_seed_off"].cpu().numpy()
    assert eo[0] == 0 and eo[-1] == n and np.all(np.diff(eo) >= 0)
    for e in range(len(eo) - 1):
        hs = gh[eo[e]:eo[e + 1]]
        if hs.size:
            assert hs.min() >= off[e] and hs.max() < off[e + 1]
    cov = got["cov"].cpu().numpy()
    assert np.all(cov[[0, 2, 5, 9, 14, 20]] > 0) and np.count_nonzero(np.delete(cov, [0, 2, 5, 9, 14, 20], 0)) == 0


def _oracle_pair(geo, xyz, layer, off, cuts):
    import oracle
    ref = oracle.seed_quads(geo, xyz, layer, off, **cuts)
    loose = oracle.seed_quads(geo, xyz, layer, off, eps=EPS, **cuts)
    # global ids from the oracle are caller ids already
    return ref, loose


def test_c2_event_equals_oracle():
    import paper_2002_06295_gb300 as mkf
    ev = sev.make_config_event(2)
    off = np.array([0, ev.n_hits])
    ctx = _ctx_for(ev)
    _bin(ctx, ev.hit_xyz, ev.hit_lcov, ev.hit_layer, off)
    got = mkf.mkf_seed_tracks(ctx, **CUTS)
    mkf.mkf_sync(ctx)
    ref, loose = _oracle_pair(ev.geom, ev.hit_xyz, ev.hit_layer, off, CUTS)
    assert got["n"] > 2000
    _compare(got, loose, ref, off)
    w = mkf.mkf_get_seed_stats(ctx)
    assert w["seeds"] == got["n"]
    assert w["pairs"] <= w["l1_examined"] and w["triplets"] <= w["l2_examined"] and w["seeds"] <= w["l3_examined"]
    assert w["pairs"] > 0 and w["triplets"] >= w["seeds"] // 4
    ctx.close()


def test_batch_of_events_equals_oracle():
    import paper_2002_06295_gb300 as mkf
    b = sev.make_batch(3, n_events=6)
    xyz, lay, lcov = b.cat("hit_xyz"), b.cat("hit_layer"), b.cat("hit_lcov")
    off = b.hit_off
    ctx = _ctx_for(b)
    _bin(ctx, xyz, lcov, lay, off)
    got = mkf.mkf_seed_tracks(ctx, **CUTS_B10)
    mkf.mkf_sync(ctx)
    ref, loose = _oracle_pair(b.geom, xyz, lay, off, CUTS_B10)
    assert got["n"] > 1000
    _compare(got, loose, ref, off)
    ctx.close()


def test_masked_hits_are_not_used():
    import paper_2002_06295_gb300 as mkf
    ev = sev.make_config_event(2, n_tracks=1500)
    off = np.array([0, ev.n_hits])
    rng = np.random.default_rng(3)
    mask = (rng.random(ev.n_hits) < 0.3).astype(np.uint8)
    ctx = _ctx_for(ev)
    _bin(ctx, ev.hit_xyz, ev.hit_lcov, ev.hit_layer, off, mask=mask)
    got = mkf.mkf_seed_tracks(ctx, **CUTS)
    mkf.mkf_sync(ctx)
    keep = np.nonzero(mask == 0)[0]
    import oracle
    ref = oracle.seed_quads(ev.geom, ev.hit_xyz[keep], ev.hit_layer[keep], **CUTS)
    loose = oracle.seed_quads(ev.geom, ev.hit_xyz[keep], ev.hit_layer[keep], eps=EPS, **CUTS)
    for r in (ref, loose):
        r["hits"] = keep[r["hits"]]
    assert got["n"] > 100
    assert not mask[got["hits"].cpu().numpy()].any()
    _compare(got, loose, ref, off)
    ctx.close()


def test_capacity_is_reported():
    import paper_2002_06295_gb300 as mkf
    ev = sev.make_config_event(2, n_tracks=500)
    ctx = _ctx_for(ev)
    _bin(ctx, ev.hit_xyz, ev.hit_lcov, ev.hit_layer, np.array([0, ev.n_hits]))
    got = mkf.mkf_seed_tracks(ctx, max_seeds=10, **CUTS)
    assert got["n"] > 10
    with pytest.raises(mkf.MkfError):
        mkf.mkf_sync(ctx)
    ctx.close()


def test_tracks_built_from_hit_seeds():
    """Building from the hit seeds finds the prompt tracks the seeds cover:
    more than 95 % of the particles with pT >= 1 GeV and a hit on each seeding
    layer give a kept track with >= 75 % of its hits from that particle."""
    import oracle
    import paper_2002_06295_gb300 as mkf
    ev = sev.make_config_event(2)
    ctx = _ctx_for(ev)
    _bin(ctx, ev.hit_xyz, ev.hit_lcov, ev.hit_layer, np.array([0, ev.n_hits]))
    s = mkf.mkf_seed_tracks(ctx, **CUTS)
    assert s["n"] > 0
    o = mkf.mkf_build_tracks(ctx, s["par"], s["cov"], s["ev_seed_off"], chi2_cut=30.0, max_cands=6, max_holes=3,
                             min_hits=4, dup_frac=0.5)
    mkf.mkf_sync(ctx)
    hits = o["hits"].cpu().numpy().reshape(s["n"], -1)
    flags = o["flags"].cpu().numpy()
    matched = set()
    for k in hits[flags == mkf.TRK_KEPT]:
        hk = k[k >= 0]
        if hk.size == 0:
            continue
        ids_t, cnt = np.unique(ev.hit_track[hk], return_counts=True)
        j = np.argmax(cnt)
        if ids_t[j] >= 0 and cnt[j] >= 0.75 * hk.size:
            matched.add(int(ids_t[j]))
    ids, _ = oracle.seeding_layers(ev.geom)
    want = [t for t in range(ev.n_seeds)
            if all((ev.true_layers[t] == l).any() for l in ids) and 1.0 / abs(ev.true_par[t, 3]) >= 1.0]
    n_ok = sum(t in matched for t in want)
    assert len(want) > 1000
    assert n_ok / len(want) > 0.95, (n_ok, len(want))
    ctx.close()


def test_event_without_layer0_hits_and_count_only():
    """A batch whose middle event has no layer-0 hits: its CSR range is empty
    and the other events match the oracle; max_seeds = 0 only counts."""
    import oracle
    import paper_2002_06295_gb300 as mkf
    evs = [sev.make_config_event(2, e, n_tracks=600) for e in range(3)]
    ids, _ = oracle.seeding_layers(evs[0].geom)
    keep = evs[1].hit_layer != ids[0]
    xyz = np.concatenate([evs[0].hit_xyz, evs[1].hit_xyz[keep], evs[2].hit_xyz])
    lay = np.concatenate([evs[0].hit_layer, evs[1].hit_layer[keep], evs[2].hit_layer])
    lcov = np.concatenate([evs[0].hit_lcov, evs[1].hit_lcov[keep], evs[2].hit_lcov])
    off = np.cumsum([0, evs[0].n_hits, int(keep.sum()), evs[2].n_hits])
    ctx = _ctx_for(evs[0])
    _bin(ctx, xyz, lcov, lay, off)
    got = mkf.mkf_seed_tracks(ctx, **CUTS)
    mkf.mkf_sync(ctx)
    eo = got["ev_seed_off"].cpu().numpy()
    assert eo[2] == eo[1] and eo[1] > 0 and eo[3] > eo[2]
    ref, loose = _oracle_pair(evs[0].geom, xyz, lay, off, CUTS)
    _compare(got, loose, ref, off)
    c = mkf.mkf_seed_tracks(ctx, max_seeds=0, **CUTS)
    assert c["n"] == got["n"]
    with pytest.raises(mkf.MkfError):
        mkf.mkf_sync(ctx)
    ctx.close()


def test_seeding_build_fit_captured_in_one_graph():
    """With a fixed triplet capacity, hit-based seeding reads nothing back, so
    binning -> seeding -> building (n_seeds = max_seeds, the count taken from
    ev_seed_off on the device) -> outward fit is captured as one CUDA graph.
    Two replays equal the synchronous path (seeding with its read-back,
    building the n seeds found, fitting them) on a six-event batch: the seeds,
    the event offsets, the built tracks and the fit; rows past n are empty
    tracks."""
    import paper_2002_06295_gb300 as mkf
    from tests._util import make_ctx
    b = sev.make_batch(3)
    evs = b.events[:6]
    xyz = np.concatenate([e.hit_xyz for e in evs])
    lcov = np.concatenate([e.hit_lcov for e in evs])
    lay = np.concatenate([e.hit_layer for e in evs])
    off = np.concatenate([[0], np.cumsum([e.n_hits for e in evs])])
    dev = torch.device("cuda", 0)
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(dev, dt)
    X, Lc, Ly, O = t(xyz.T, torch.float32), t(lcov.T, torch.float32), t(lay, torch.int32), t(off, torch.int64)
    kw = dict(chi2_cut=30.0, max_cands=4, max_holes=3, min_hits=4, dup_frac=0.5)
    cap_seeds = 200000
    # synchronous path
    ctx = make_ctx(b.geom)
    mkf.mkf_bin_hits(ctx, X, Lc, Ly, O)
    s0 = mkf.mkf_seed_tracks(ctx, max_seeds=cap_seeds, **CUTS_B10)
    n = s0["n"]
    assert 1000 < n < cap_seeds
    b0 = mkf.mkf_build_tracks(ctx, s0["par"].contiguous(), s0["cov"].contiguous(), s0["ev_seed_off"], **kw)
    f0 = mkf.mkf_fit_tracks(ctx, X, Lc, Ly, b0["hits"], s0["par"].contiguous(), s0["cov"].contiguous())
    mkf.mkf_sync(ctx)
    ref = {k: v.cpu().numpy() for k, v in b0.items()}
    fref = {k: v.cpu().numpy() for k, v in f0.items()}
    seeds_ref = (s0["par"].cpu().numpy(), s0["hits"].cpu().numpy(), s0["ev_seed_off"].cpu().numpy())
    # fixed capacity, no read-back: one graph
    mkf.mkf_set_seed_config(ctx, 4 * int(off[-1]))
    sbuf = dict(par=torch.zeros(6 * cap_seeds, device=dev), cov=torch.zeros(21 * cap_seeds, device=dev),
                hits=torch.zeros(4 * cap_seeds, dtype=torch.int32, device=dev),
                ev_seed_off=torch.zeros(len(evs) + 1, dtype=torch.int64, device=dev))
    bout = mkf.alloc_build_outputs(ctx, cap_seeds)
    fout = dict(par=torch.empty((6, cap_seeds), device=dev), cov=torch.empty((21, cap_seeds), device=dev),
                chi2=torch.empty(cap_seeds, device=dev), ok=torch.empty(cap_seeds, dtype=torch.int32, device=dev))

    def step():
        mkf.mkf_bin_hits(ctx, X, Lc, Ly, O)
        s = mkf.mkf_seed_tracks(ctx, out=sbuf, read_count=False, **CUTS_B10)
        mkf.mkf_build_tracks(ctx, s["par"], s["cov"], s["ev_seed_off"], out=bout, **kw)
        mkf.mkf_fit_tracks(ctx, X, Lc, Ly, bout["hits"], s["par"], s["cov"], out=fout)

    step()   # sizes the workspace outside the capture
    torch.cuda.synchronize()
    mkf.mkf_sync(ctx)
    mkf.mkf_set_timing(ctx, False)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step()
    for _ in range(2):
        for v in bout.values():
            v.fill_(7)
        g.replay()
        torch.cuda.synchronize()
        mkf.mkf_sync(ctx)
        assert np.array_equal(sbuf["ev_seed_off"].cpu().numpy(), seeds_ref[2])
        par = sbuf["par"].view(6, cap_seeds).cpu().numpy()
        assert np.array_equal(par[:, :n], seeds_ref[0])
        assert np.array_equal(sbuf["hits"].view(cap_seeds, 4).cpu().numpy()[:n], seeds_ref[1])
        got = {k: v.cpu().numpy() for k, v in bout.items()}
        for k in ("hits", "flags", "score"):
            assert np.array_equal(got[k][:n], ref[k]), k
        assert np.array_equal(got["par"][:, :n], ref["par"])
        assert (got["hits"][n:] == -1).all() and (got["flags"][n:] == mkf.TRK_SHORT).all()
        fgot = {k: v.cpu().numpy() for k, v in fout.items()}
        assert np.array_equal(fgot["par"][:, :n], fref["par"])
        assert np.array_equal(fgot["chi2"][:n], fref["chi2"])
    ctx.close()
