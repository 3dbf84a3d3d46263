"""The fits and the fit adjoint on degenerate inputs, through the C ABI,
against the oracle: no tracks at all, and rows with no listed hit, a single
hit, only the outermost hit, every other hit missing, and the first hits
missing.  Same bars as the full-row tests: parameters and covariances 1e-4,
chi2 1e-3 relative (1e-3 absolute below chi2 = 1), gradient components 1e-3
of themselves above their FP32 floor."""
import numpy as np
import pytest
import torch

from _util import CHI2_RTOL, COV_RTOL, PAR_RTOL, cov_rel_err, f32, i32, make_ctx, par_rel_err
from test_gpu_adjoint import GRAD_RTOL, _component_errors, _floors, _inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _thin_rows(hits):
    """Rows 0-9 empty, 10-19 the first hit only, 20-29 the last hit only,
    30-59 every other hit, 60-89 without their first three hits; the rest
    whole."""
    h = hits.copy()
    h[0:10] = -1
    h[10:20, 1:] = -1
    h[20:30, :-1] = -1
    h[30:60, 1::2] = -1
    h[60:90, :3] = -1
    return h


def _np(t):
    return t.cpu().numpy().astype(np.float64)


def test_fits_of_no_tracks():
    import paper_2002_06295_gb300 as mkf
    g, ev, hits, sp, sc, align, x0, up = _inputs(n=50)
    dev = torch.device("cuda", 0)
    ctx = make_ctx(g)
    K = hits.shape[1]
    xyz, lcov, lay = f32(ev.hit_xyz.T, dev), f32(ev.hit_lcov.T, dev), i32(ev.hit_layer, dev)
    h0 = torch.zeros((0, K), dtype=torch.int32, device=dev)
    p0 = torch.zeros((6, 0), dtype=torch.float32, device=dev)
    c0 = torch.zeros((21, 0), dtype=torch.float32, device=dev)
    ck = torch.zeros((K, 27, 0), dtype=torch.float32, device=dev)
    o = mkf.mkf_fit_tracks(ctx, xyz, lcov, lay, h0, p0, c0, ckpt=ck)
    b = mkf.mkf_fit_backward(ctx, xyz, lcov, lay, h0, p0)
    g0 = torch.zeros(0, dtype=torch.float32, device=dev)
    a = mkf.mkf_fit_tracks_adjoint(ctx, xyz, lcov, lay, h0, p0, c0, ck, g_chi2=g0)
    mkf.mkf_sync(ctx)
    assert o["par"].shape == (6, 0) and b["cov"].shape == (21, 0)
    # no tracks: every gradient is zero (the outputs start from garbage)
    assert (a["g_hit"] == 0).all() and (a["g_align"] == 0).all() and (a["g_x0"] == 0).all()
    ctx.close()


def test_fits_of_thin_rows():
    import oracle
    import paper_2002_06295_gb300 as mkf
    g, ev, hits, sp, sc, align, x0, up = _inputs(n=400, seed=33)
    hits = _thin_rows(hits)
    geo = oracle.Geo.of(g)
    dev = torch.device("cuda", 0)
    ctx = make_ctx(g)
    T, K = hits.shape
    xyz, lcov, lay, hd = f32(ev.hit_xyz.T, dev), f32(ev.hit_lcov.T, dev), i32(ev.hit_layer, dev), i32(hits, dev)
    al, xx = f32(align, dev), f32(x0, dev)
    ckpt = torch.empty((K, 27, T), dtype=torch.float32, device=dev)
    o = mkf.mkf_fit_tracks(ctx, xyz, lcov, lay, hd, f32(sp.T, dev), f32(sc.T, dev), align=al, x0=xx, ckpt=ckpt)
    mkf.mkf_sync(ctx)
    par, cov, chi2, ok = oracle.fit(geo, ev.hit_xyz, ev.hit_lcov, ev.hit_layer, hits, sp, sc, align=align, x0=x0)
    gp, gc, gx = _np(o["par"]).T, _np(o["cov"]).T, _np(o["chi2"])
    assert ok.all() and (o["ok"].cpu().numpy() >= 1).all()
    pe, ce = par_rel_err(gp, par), cov_rel_err(gc, cov)
    print("thin rows, forward: par", pe.max(), "cov", ce.max())
    assert pe.max() < PAR_RTOL and ce.max() < COV_RTOL
    assert (np.abs(gx - chi2) <= CHI2_RTOL * chi2).all()
    assert (gx[:10] == 0).all()
    assert np.array_equal(_np(o["par"]).T[:10], sp[:10].astype(np.float32))

    # inward, both from the oracle's outward result rounded to FP32 (with the
    # 100x prior a row's single hit gives chi2 ~1e-6, which the rounding of a
    # start given in FP64 to one side only would decide)
    parq = np.asarray(par, np.float32).astype(np.float64)
    b = mkf.mkf_fit_backward(ctx, xyz, lcov, lay, hd, f32(parq.T, dev), align=al, x0=xx)
    mkf.mkf_sync(ctx)
    bpar, bcov, bchi2, bok = oracle.fit(geo, ev.hit_xyz, ev.hit_lcov, ev.hit_layer, hits, parq, cov, align=align,
                                        x0=x0, direction=-1)
    gp, gc, gx = _np(b["par"]).T, _np(b["cov"]).T, _np(b["chi2"])
    assert bok.all() and (b["ok"].cpu().numpy() == 1).all()
    pe, ce = par_rel_err(gp, bpar), cov_rel_err(gc, bcov)
    print("thin rows, inward: par", pe.max(), "cov", ce.max())
    assert pe.max() < PAR_RTOL and ce.max() < COV_RTOL
    # a chi2 far below one degree of freedom (a single hit against the prior)
    # is held to 1e-3 of one: its relative error is that of its tiny residual
    bad = np.nonzero(np.abs(gx - bchi2) > CHI2_RTOL * np.maximum(bchi2, 1.0))[0]
    print("thin rows, inward chi2: rows below 1:", np.nonzero(bchi2 < 1)[0][:20])
    assert len(bad) == 0, list(zip(bad[:8], gx[bad[:8]], bchi2[bad[:8]]))

    # adjoint of the outward fit
    gd = {k: f32(v.T if v.ndim == 2 else v, dev) for k, v in up.items()}
    a = mkf.mkf_fit_tracks_adjoint(ctx, xyz, lcov, lay, hd, f32(sp.T, dev), f32(sc.T, dev), ckpt, align=al, x0=xx,
                                   **gd)
    mkf.mkf_sync(ctx)
    rh, ra, rx = oracle.fit_grad(geo, ev.hit_xyz, ev.hit_lcov, ev.hit_layer, hits, sp, sc, up["g_chi2"],
                                 g_par=up["g_par"], g_cov=up["g_cov"], align=align, x0=x0)
    gh, ga, gxx = _np(a["g_hit"]).T, _np(a["g_align"]), _np(a["g_x0"])
    used = np.unique(hits[hits >= 0])
    unused = np.setdiff1d(np.arange(ev.n_hits), used)
    assert (gh[unused] == 0).all()
    f_hit, f_layer, f_x0 = _floors(g, ev, hits, sp, sc, up, align, x0)
    report = {}
    for name, x, y, f in (("hit", gh[used], rh[used], f_hit), ("align", ga, ra, f_layer), ("x0", gxx, rx, f_x0)):
        report[name] = _component_errors(x, y, f)
    print("thin rows, adjoint (worst component / its bound, norm-wise):", report)
    for name, (worst, enorm) in report.items():
        assert enorm < GRAD_RTOL, (name, report)
        assert worst <= 1.0, (name, report)
    ctx.close()
