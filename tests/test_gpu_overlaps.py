"""Overlap-hit recovery on the GPU (Sec. 3, hits in overlapping modules)
against the FP64 oracle, on a CMS-like event whose barrel crossings leave a
second hit 30 % of the time; both sides see the same float32 inputs.

An overlap hit's chi2 is formed from residuals of tens of microns between
positions of up to R_max ~ 110 cm that carry FP32 rounding, ~4 eps R_max
(eps = 2^-24) each, so the FP32 chi2 of a residual r/sigma carries
2 sqrt(chi2) d + d^2 with d = 4 eps R_max / sigma_min on top of its 1e-3
relative bar.  A slot's choice is compared exactly where the oracle's choice
is clear of that: its best chi2 more than 1e-3 (plus that error) away from the
cut and below the runner-up.

Every track is compared.  The tracks whose fit fails (chi2/ndf > 5: central
loopers that reach the disks only after several turns, and forward tracks
whose seed theta is off by a large fraction of theta, where one linearised
pass cannot follow the helix) have states that FP32 and FP64 carry apart; on
them at most 0.5 % of the clear slots may differ, and every other track must
agree on every clear slot.  Also: tracks built on the GPU recover the
simulation's overlap hits, and the work counters add up."""
import numpy as np
import pytest
import torch

import synth.events as sev

pytestmark = pytest.mark.gpu
CUT = 20.0


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


EPS32 = 2.0 ** -24


@pytest.fixture(scope="module")
def event():
    ev = sev.make_config_event(2, overlap_frac=0.3)
    q = lambda a: np.asarray(a, np.float32).astype(np.float64)
    ev.hit_xyz, ev.hit_lcov = q(ev.hit_xyz), q(ev.hit_lcov)
    ev.seed_par, ev.seed_cov = q(ev.seed_par), q(ev.seed_cov)
    return ev


def _setup(ev):
    from tests._util import make_ctx, f32, i32, i64
    import paper_2002_06295_gb300 as mkf
    dev = torch.device("cuda", 0)
    ctx = make_ctx(ev.geom)
    d = dict(xyz=f32(ev.hit_xyz.T, dev), lcov=f32(ev.hit_lcov.T, dev), layer=i32(ev.hit_layer, dev))
    mkf.mkf_bin_hits(ctx, d["xyz"], d["lcov"], d["layer"], i64(np.array([0, ev.n_hits]), dev))
    return ctx, d, dev


def test_true_tracks_equal_oracle(event):
    import oracle
    import paper_2002_06295_gb300 as mkf
    from tests._util import f32, i32
    ev = event
    sel = np.array([t for t in range(ev.n_seeds) if (ev.true_hits[t] >= 0).sum() >= 6])
    hits = ev.true_hits[sel].astype(np.int32)
    ctx, d, dev = _setup(ev)
    o = mkf.mkf_find_overlaps(ctx, d["xyz"], d["lcov"], d["layer"], i32(hits, dev), f32(ev.seed_par[sel].T, dev),
                              f32(ev.seed_cov[sel].T, dev), chi2_cut=CUT)
    mkf.mkf_sync(ctx)
    gh, gc = o["hit"].cpu().numpy(), o["chi2"].cpu().numpy()
    ref = oracle.overlaps(oracle.Geo.of(ev.geom), ev.hit_xyz, ev.hit_lcov, ev.hit_layer, hits, ev.seed_par[sel],
                          ev.seed_cov[sel], chi2_cut=CUT)
    slots = hits >= 0
    best = ref["best"]
    assert not (best < 0).any()   # the Joseph-form oracle keeps every R positive
    r_max = float(np.abs(ev.geom.table()[:, 1:4]).max())
    d = 4 * EPS32 * r_max / np.sqrt(ev.hit_lcov[:, :2].min())
    chi2_err = lambda c: 1e-3 * c + 2 * np.sqrt(np.maximum(c, 0)) * d + d * d
    # clear: no candidate near the cut, or a clear winner below it
    clear = slots & ((best > CUT + chi2_err(CUT)) | ((best < CUT - chi2_err(CUT)) & (ref["gap"] * best > 2 * chi2_err(best))))
    assert clear.sum() > 0.99 * slots.sum()
    _, _, fchi2, fok = oracle.fit(oracle.Geo.of(ev.geom), ev.hit_xyz, ev.hit_lcov, ev.hit_layer, hits,
                                  ev.seed_par[sel], ev.seed_cov[sel])
    failed = (fok != 1) | (fchi2 > 5.0 * 2 * slots.sum(1))
    assert failed.mean() < 0.06
    same = gh == ref["hit"]
    assert same[clear & ~failed[:, None]].all()
    assert (~same[clear & failed[:, None]]).sum() <= 0.005 * (clear & failed[:, None]).sum()
    found = clear & (ref["hit"] >= 0) & same
    assert found.sum() > 1000
    assert np.all(np.abs(gc[found] - ref["chi2"][found]) <= chi2_err(ref["chi2"][found]))
    assert np.all(gh[~slots] == -1)
    w = mkf.mkf_get_overlap_stats(ctx)
    assert w["found"] == int((gh >= 0).sum()) and w["hits_fitted"] <= int(slots.sum())
    assert w["hits_fitted"] > 0.99 * slots.sum() and w["candidates"] >= w["found"]
    ctx.close()


def test_built_tracks_recover_simulated_overlaps(event):
    import paper_2002_06295_gb300 as mkf
    from tests._util import f32, i64
    ev = event
    ctx, d, dev = _setup(ev)
    sp, sc = f32(ev.seed_par.T, dev), f32(ev.seed_cov.T, dev)
    b = mkf.mkf_build_tracks(ctx, sp, sc, i64(np.array([0, ev.n_seeds]), dev), chi2_cut=30.0, max_cands=6,
                             max_holes=3, min_hits=4, dup_frac=0.5)
    o = mkf.mkf_find_overlaps(ctx, d["xyz"], d["lcov"], d["layer"], b["hits"], sp, sc, chi2_cut=CUT)
    mkf.mkf_sync(ctx)
    bh, flags, gh = b["hits"].cpu().numpy(), b["flags"].cpu().numpy(), o["hit"].cpu().numpy()
    # crossings where the built track took the true hit and the simulation left an overlap hit
    ok = tot = fake = n_plain = 0
    for t in np.nonzero(flags == mkf.TRK_KEPT)[0]:
        truth = {int(h): k for k, h in enumerate(ev.true_hits[t]) if h >= 0}
        for k, h in enumerate(bh[t]):
            if h < 0 or int(h) not in truth:
                continue
            ov = ev.true_overlap[t, truth[int(h)]]
            if ov >= 0:
                tot += 1
                ok += gh[t, k] == ov
            else:
                n_plain += 1
                fake += gh[t, k] >= 0
    assert tot > 2000
    assert ok / tot > 0.95, (ok, tot)
    assert fake / n_plain < 0.05, (fake, n_plain)
    ctx.close()


def test_no_tracks_and_tracks_without_hits(event):
    import paper_2002_06295_gb300 as mkf
    ev = event
    ctx, d, dev = _setup(ev)
    z = torch.zeros((0, 38), dtype=torch.int32, device=dev)
    o = mkf.mkf_find_overlaps(ctx, d["xyz"], d["lcov"], d["layer"], z, torch.zeros((6, 0), device=dev),
                              torch.zeros((21, 0), device=dev))
    assert o["hit"].numel() == 0
    h = torch.full((3, 38), -1, dtype=torch.int32, device=dev)
    sp = torch.tensor(ev.seed_par[:3].T.copy(), dtype=torch.float32, device=dev)
    sc = torch.tensor(ev.seed_cov[:3].T.copy(), dtype=torch.float32, device=dev)
    o = mkf.mkf_find_overlaps(ctx, d["xyz"], d["lcov"], d["layer"], h, sp, sc)
    mkf.mkf_sync(ctx)
    assert (o["hit"].cpu().numpy() == -1).all()
    ctx.close()


def test_same_in_every_launch_shape(event):
    """One thread per track in blocks of 32, 64 or 128 by track count, and
    eight lanes per track: copies of the same tracks find the same overlap
    hits with the same chi2, bit for bit, in every shape."""
    import paper_2002_06295_gb300 as mkf
    from tests._util import f32, i32
    ev = event
    sel = np.array([t for t in range(ev.n_seeds) if (ev.true_hits[t] >= 0).sum() >= 6])[:1200]
    hits = ev.true_hits[sel].astype(np.int32)
    n = hits.shape[0]
    ctx, d, dev = _setup(ev)
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    outs = {}
    for lanes in (1, 8):
        mkf.mkf_set_overlap_config(ctx, lanes)
        for copies in (1, (n_sm * 64) // n + 1, (n_sm * 128) // n + 1):
            o = mkf.mkf_find_overlaps(ctx, d["xyz"], d["lcov"], d["layer"], i32(np.tile(hits, (copies, 1)), dev),
                                      f32(np.tile(ev.seed_par[sel], (copies, 1)).T, dev),
                                      f32(np.tile(ev.seed_cov[sel], (copies, 1)).T, dev), chi2_cut=CUT)
            mkf.mkf_sync(ctx)
            outs[(lanes, copies)] = (o["hit"].cpu().numpy(), o["chi2"].cpu().numpy())
    with pytest.raises(mkf.MkfError):
        mkf.mkf_set_overlap_config(ctx, 4)
    bh, bc = outs[(1, 1)]
    assert (bh >= 0).sum() > 0
    for (lanes, copies), (h, c) in outs.items():
        for k in range(copies):
            rows = slice(k * n, (k + 1) * n)
            assert np.array_equal(h[rows], bh), copies
            assert np.array_equal(c[rows], bc, equal_nan=True), copies
    ctx.close()
