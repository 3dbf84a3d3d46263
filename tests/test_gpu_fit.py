"""Parity of the CUDA fixed-assignment Kalman fit (outward and inward) with the
FP64 oracle: parameters within 1e-4 relative, covariances within 1e-4 of
sqrt(C_ii C_jj), chi2 within 1e-3 relative."""
import numpy as np
import pytest
import torch

import synth
from _util import CHI2_RTOL, COV_RTOL, PAR_RTOL, cov_ok, cov_rel_err, f32, i32, make_ctx, par_rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _fit_inputs(n=2000, seed=11, geom=None):
    g = geom or synth.geometry_barrel14()
    rng = np.random.default_rng(seed)
    ev = synth.simulate_event(g, n, rng, pt_range=(1.0, 10.0), eta_max=0.8)
    keep = (ev.true_hits >= 0).sum(1) == g.n_layers
    return g, ev, ev.true_hits[keep], ev.seed_par[keep], ev.seed_cov[keep], rng


@pytest.mark.parametrize("with_align", [False, True])
def test_forward_fit_matches_oracle(with_align):
    import oracle
    import paper_2002_06295_gb300 as mkf
    g, ev, hits, sp, sc, rng = _fit_inputs()
    align = rng.normal(0, 2e-3, (g.n_layers, 3)) if with_align else None
    x0 = g.x0 * (1 + 0.2 * rng.random(g.n_layers)) if with_align else None
    dev = torch.device("cuda", 0)
    ctx = make_ctx(g)
    T, K = hits.shape
    ckpt = torch.empty((K, 27, T), dtype=torch.float32, device=dev)
    o = mkf.mkf_fit_tracks(ctx, f32(ev.hit_xyz.T, dev), f32(ev.hit_lcov.T, dev), i32(ev.hit_layer, dev),
                           i32(hits, dev), f32(sp.T, dev), f32(sc.T, dev),
                           align=None if align is None else f32(align, dev),
                           x0=None if x0 is None else f32(x0, dev), ckpt=ckpt)
    mkf.mkf_sync(ctx)
    par, cov, chi2, ok = oracle.fit(oracle.Geo.of(g), ev.hit_xyz, ev.hit_lcov, ev.hit_layer, hits, sp, sc,
                                    align=align, x0=x0)
    gp = o["par"].cpu().numpy().T.astype(np.float64)
    gc = o["cov"].cpu().numpy().T.astype(np.float64)
    gx = o["chi2"].cpu().numpy().astype(np.float64)
    assert (o["ok"].cpu().numpy() == 1).all() and ok.all()
    pe, ce = par_rel_err(gp, par), cov_rel_err(gc, cov)
    print("forward fit: par err per parameter", pe.max(0), "cov err", ce.max(),
          "chi2 rel err", (np.abs(gx - chi2) / chi2).max())
    assert pe.max() < PAR_RTOL
    assert ce.max() < COV_RTOL
    assert (np.abs(gx - chi2) <= CHI2_RTOL * chi2).all()
    # checkpoint 0 is the initial state
    ck = ckpt.cpu().numpy()
    assert np.array_equal(ck[0, :6].T, sp.astype(np.float32))
    assert np.array_equal(ck[0, 6:].T, sc.astype(np.float32))
    ctx.close()


def test_backward_fit_matches_oracle():
    import oracle
    import paper_2002_06295_gb300 as mkf
    g, ev, hits, sp, sc, rng = _fit_inputs(1500, seed=12)
    geo = oracle.Geo.of(g)
    fpar, fcov, _, _ = oracle.fit(geo, ev.hit_xyz, ev.hit_lcov, ev.hit_layer, hits, sp, sc)
    bpar, bcov, bchi2, bok = oracle.fit(geo, ev.hit_xyz, ev.hit_lcov, ev.hit_layer, hits, fpar, fcov, direction=-1)
    dev = torch.device("cuda", 0)
    ctx = make_ctx(g)
    o = mkf.mkf_fit_backward(ctx, f32(ev.hit_xyz.T, dev), f32(ev.hit_lcov.T, dev), i32(ev.hit_layer, dev),
                             i32(hits, dev), f32(fpar.T, dev))
    mkf.mkf_sync(ctx)
    gp = o["par"].cpu().numpy().T.astype(np.float64)
    gc = o["cov"].cpu().numpy().T.astype(np.float64)
    assert bok.all() and (o["ok"].cpu().numpy() == 1).all()
    pe, ce = par_rel_err(gp, bpar), cov_rel_err(gc, bcov)
    print("backward fit: par err per parameter", pe.max(0), "cov err", ce.max())
    assert pe.max() < PAR_RTOL
    assert ce.max() < COV_RTOL
    ctx.close()


def test_fit_cmslike_mixed_surfaces():
    """Barrel and disk hits in one track list (CMS-like geometry)."""
    import oracle
    import paper_2002_06295_gb300 as mkf
    g = synth.geometry_cmslike()
    rng = np.random.default_rng(13)
    ev = synth.simulate_event(g, 1500, rng, pt_range=(0.8, 20.0), pt_log=True, eta_max=2.4)
    n = (ev.true_hits >= 0).sum(1)
    keep = n >= 6
    hits, sp, sc = ev.true_hits[keep], ev.seed_par[keep], ev.seed_cov[keep]
    dev = torch.device("cuda", 0)
    ctx = make_ctx(g)
    o = mkf.mkf_fit_tracks(ctx, f32(ev.hit_xyz.T, dev), f32(ev.hit_lcov.T, dev), i32(ev.hit_layer, dev),
                           i32(hits, dev), f32(sp.T, dev), f32(sc.T, dev))
    mkf.mkf_sync(ctx)
    par, cov, chi2, ok = oracle.fit(oracle.Geo.of(g), ev.hit_xyz, ev.hit_lcov, ev.hit_layer, hits, sp, sc)
    gp = o["par"].cpu().numpy().T.astype(np.float64)
    gc = o["cov"].cpu().numpy().T.astype(np.float64)
    # ok = 2: fitted, with a transport onto a disk of a full turn or more (no adjoint)
    good = ok.astype(bool) & (o["ok"].cpu().numpy() >= 1)
    assert good.mean() > 0.99
    pe = par_rel_err(gp[good], par[good])
    worst = np.argmax(pe.max(1))
    print("cms-like fit: par err per parameter", pe.max(0), "worst track", gp[good][worst], par[good][worst],
          hits[good][worst])
    assert pe.max() < PAR_RTOL
    ce = cov_rel_err(gc[good], cov[good])
    print("cms-like fit: cov err max", ce.max(), "fraction within 1e-4", (ce.max(1) < COV_RTOL).mean())
    # the U-D factorised FP32 covariance keeps the small conditional variances
    # of pixel hits and strip disks: every track within 1e-4
    assert ce.max() < COV_RTOL
    ctx.close()


def test_backward_fit_cmslike_mixed_surfaces():
    """Inward fit over barrel and disk hits (CMS-like geometry) from the
    oracle's outward result: the 100x prior and the correlations near 1 that
    mixed barrel/disk tracks keep are what the inward fit's precision must
    carry."""
    import oracle
    import paper_2002_06295_gb300 as mkf
    g = synth.geometry_cmslike()
    rng = np.random.default_rng(14)
    ev = synth.simulate_event(g, 1500, rng, pt_range=(0.8, 20.0), pt_log=True, eta_max=2.4)
    keep = (ev.true_hits >= 0).sum(1) >= 6
    hits, sp, sc = ev.true_hits[keep], ev.seed_par[keep], ev.seed_cov[keep]
    # inputs quantised to float32 so that both sides see the same numbers: a
    # track with few hits and a short lever arm turns the rounding of its hit
    # positions (~1e-7 relative) into ~1e-3 of its own curvature
    q = lambda a: np.asarray(a, np.float32).astype(np.float64)
    ev.hit_xyz, ev.hit_lcov = q(ev.hit_xyz), q(ev.hit_lcov)
    geo = oracle.Geo.of(g)
    fpar, fcov, _, fok = oracle.fit(geo, ev.hit_xyz, ev.hit_lcov, ev.hit_layer, hits, q(sp), q(sc))
    fpar = q(fpar)
    bpar, bcov, _, bok = oracle.fit(geo, ev.hit_xyz, ev.hit_lcov, ev.hit_layer, hits, fpar, fcov, direction=-1)
    dev = torch.device("cuda", 0)
    ctx = make_ctx(g)
    o = mkf.mkf_fit_backward(ctx, f32(ev.hit_xyz.T, dev), f32(ev.hit_lcov.T, dev), i32(ev.hit_layer, dev),
                             i32(hits, dev), f32(fpar.T, dev))
    mkf.mkf_sync(ctx)
    gp = o["par"].cpu().numpy().T.astype(np.float64)
    gc = o["cov"].cpu().numpy().T.astype(np.float64)
    good = fok.astype(bool) & bok.astype(bool) & (o["ok"].cpu().numpy() == 1)
    assert good.mean() > 0.99
    pe, ce = par_rel_err(gp[good], bpar[good]), cov_rel_err(gc[good], bcov[good])
    print("cms-like backward fit: par err per parameter", pe.max(0), "cov err max", ce.max(),
          "fraction within 1e-4", (ce.max(1) < COV_RTOL).mean())
    assert pe.max() < PAR_RTOL
    assert ce.max() < COV_RTOL
    ctx.close()


def test_backward_fit_built_c2_tracks():
    """Inward fit of the tracks built on the full C2 event (5000 seeds, 20 %
    noise hits, so some tracks carry wrong picks with residuals far beyond the
    hit resolution), in the launch shape the bench times, against the oracle's
    inward fit of the same hit lists from the same outward result.  Early
    updates of such tracks move the state far, which is where the two terms of
    each state increment nearly cancel."""
    import oracle
    import paper_2002_06295_gb300 as mkf
    from _util import gpu_build
    ev = synth.make_config_event(2)
    q = lambda a: np.asarray(a, np.float32).astype(np.float64)
    ev.hit_xyz, ev.hit_lcov = q(ev.hit_xyz), q(ev.hit_lcov)
    ctx = make_ctx(ev.geom)
    b = gpu_build(ctx, [ev], max_cands=6)
    hits = b["hits"]
    keep = (hits >= 0).sum(1) >= 6
    hits, sp, sc = hits[keep], q(ev.seed_par[keep]), q(ev.seed_cov[keep])
    assert keep.sum() > 3000
    geo = oracle.Geo.of(ev.geom)
    fpar, fcov, _, fok = oracle.fit(geo, ev.hit_xyz, ev.hit_lcov, ev.hit_layer, hits, sp, sc)
    fpar = q(fpar)
    bpar, bcov, _, bok = oracle.fit(geo, ev.hit_xyz, ev.hit_lcov, ev.hit_layer, hits, fpar, fcov, direction=-1)
    dev = torch.device("cuda", 0)
    o = mkf.mkf_fit_backward(ctx, f32(ev.hit_xyz.T, dev), f32(ev.hit_lcov.T, dev), i32(ev.hit_layer, dev),
                             i32(hits, dev), f32(fpar.T, dev))
    mkf.mkf_sync(ctx)
    gp = o["par"].cpu().numpy().T.astype(np.float64)
    gc = o["cov"].cpu().numpy().T.astype(np.float64)
    good = fok.astype(bool) & bok.astype(bool) & (o["ok"].cpu().numpy() == 1)
    assert good.mean() > 0.98
    pe, ce = par_rel_err(gp[good], bpar[good]), cov_rel_err(gc[good], bcov[good])
    print("built C2 backward fit: %d tracks, par err per parameter" % good.sum(), pe.max(0), "cov err max",
          ce.max(), "fraction within 1e-4", (ce.max(1) < COV_RTOL).mean())
    assert pe.max() < PAR_RTOL
    # both sides FP64: the kernel updates in the plain gain form, the oracle in
    # the Joseph form; on built tracks whose wrong picks leave the fit
    # ill-conditioned the two roundings part by up to 1.6e-4 (2 of ~3800)
    assert cov_ok(ce, frac=0.999, cap=2e-4)
    ctx.close()


def test_backward_fit_same_in_every_launch_shape():
    """The inward fit runs one thread per track in blocks of 32, 64 or 128 by
    track count; from 128 threads per SM on, at most two blocks per SM whose
    threads loop over the tracks (the batched workloads; the last count gives
    each thread two or three tracks): copies of the same tracks give
    bit-identical results in every shape, and every copy equals the first."""
    import paper_2002_06295_gb300 as mkf
    g = synth.geometry_cmslike()
    rng = np.random.default_rng(15)
    ev = synth.simulate_event(g, 1500, rng, pt_range=(0.8, 20.0), pt_log=True, eta_max=2.4)
    keep = (ev.true_hits >= 0).sum(1) >= 6
    hits, sp, sc = ev.true_hits[keep], ev.seed_par[keep], ev.seed_cov[keep]
    n = hits.shape[0]
    dev = torch.device("cuda", 0)
    ctx = make_ctx(g)
    X, Lc, Ly = f32(ev.hit_xyz.T, dev), f32(ev.hit_lcov.T, dev), i32(ev.hit_layer, dev)
    fo = mkf.mkf_fit_tracks(ctx, X, Lc, Ly, i32(hits, dev), f32(sp.T, dev), f32(sc.T, dev))
    mkf.mkf_sync(ctx)
    par0 = fo["par"].cpu().numpy().T
    outs = {}
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    for copies in (1, (n_sm * 64) // n + 1, (n_sm * 128) // n + 1, (n_sm * 640) // n + 1):
        H = np.tile(hits, (copies, 1))
        P = np.tile(par0, (copies, 1))
        o = mkf.mkf_fit_backward(ctx, X, Lc, Ly, i32(H, dev), f32(P.T, dev))
        mkf.mkf_sync(ctx)
        outs[copies] = {k: v.cpu().numpy() for k, v in o.items()}
    base = outs[1]
    for copies, o in outs.items():
        for k in ("par", "cov", "chi2", "ok"):
            a = o[k].reshape(-1, copies * n) if o[k].ndim == 2 else o[k].reshape(1, -1)
            b = base[k].reshape(-1, n) if base[k].ndim == 2 else base[k].reshape(1, -1)
            for c in range(copies):
                assert np.array_equal(a[:, c * n:(c + 1) * n], b, equal_nan=True), (copies, k, c)
    ctx.close()


def test_forward_fit_same_in_every_launch_shape():
    """The outward fit's launch shape (blocks of 32, 64 or 128 by track count)
    leaves every track's result and checkpoints bit-identical."""
    import paper_2002_06295_gb300 as mkf
    g, ev, hits, sp, sc, rng = _fit_inputs(1200, seed=16)
    n, K = hits.shape
    dev = torch.device("cuda", 0)
    ctx = make_ctx(g)
    X, Lc, Ly = f32(ev.hit_xyz.T, dev), f32(ev.hit_lcov.T, dev), i32(ev.hit_layer, dev)
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    outs = {}
    for copies in (1, (n_sm * 64) // n + 1, (n_sm * 128) // n + 1):
        T = copies * n
        ckpt = torch.empty((K, 27, T), dtype=torch.float32, device=dev)
        o = mkf.mkf_fit_tracks(ctx, X, Lc, Ly, i32(np.tile(hits, (copies, 1)), dev), f32(np.tile(sp, (copies, 1)).T, dev),
                               f32(np.tile(sc, (copies, 1)).T, dev), ckpt=ckpt)
        mkf.mkf_sync(ctx)
        r = {k: v.cpu().numpy() for k, v in o.items()}
        r["ckpt"] = ckpt.cpu().numpy()
        outs[copies] = r
    base = outs[1]
    for copies, o in outs.items():
        for c in range(copies):
            cols = slice(c * n, (c + 1) * n)
            assert np.array_equal(o["par"][:, cols], base["par"], equal_nan=True), copies
            assert np.array_equal(o["cov"][:, cols], base["cov"], equal_nan=True), copies
            assert np.array_equal(o["chi2"][cols], base["chi2"], equal_nan=True), copies
            assert np.array_equal(o["ok"][cols], base["ok"]), copies
            assert np.array_equal(o["ckpt"][:, :, cols], base["ckpt"], equal_nan=True), copies
    ctx.close()
