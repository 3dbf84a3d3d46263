"""The hand-written adjoint of the Kalman fit (through the C ABI and through
torch.autograd) against the oracle's dual-number gradient and FP64 central
finite differences (h = 1e-6).

Each gradient component g is compared with its FP64 value r on its own:
|g - r| <= 1e-3 |r| + f, where f is the error that FP32 positions alone put
into a component.  A residual is a difference of positions of up to R_max
(~100 cm) that carry FP32 rounding, so it is off by up to ~4 eps R_max
(eps = 2^-24, the hit and the propagated state each rounded about twice), and
d chi2 / d x = 2 r / sigma^2 inherits 2 (4 eps R_max) / sigma_min^2: the
hit-gradient floor f_hit = 8 eps R_max / sigma_min^2 (0.5 /cm for 100 um hits
at 100 cm).  A layer's alignment or thickness gradient is a sum of the
tracks' terms T_t, often with strong cancellation; each term carries FP32
error of ~1e-5 of itself, so the sum's floor is 1e-4 sum_t |T_t| (the terms
come from the oracle, one track at a time), and no less than f_hit sqrt(n)
for n tracks (times the layer radius for the azimuthal shift, whose lever
arm it is).  Above the floor the bar is 1e-3 relative, per component; the
norm-wise error of each group is also held to 1e-3."""
import numpy as np
import pytest
import torch

import synth
from _util import f32, i32, make_ctx

pytestmark = pytest.mark.gpu

GRAD_RTOL = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _inputs(n=300, seed=21, geom=None, pt=(1.0, 10.0), eta=0.8):
    g = geom or synth.geometry_barrel14()
    rng = np.random.default_rng(seed)
    ev = synth.simulate_event(g, n, rng, pt_range=pt, eta_max=eta)
    keep = (ev.true_hits >= 0).sum(1) >= min(g.n_layers, 6)
    hits, sp, sc = ev.true_hits[keep], ev.seed_par[keep], ev.seed_cov[keep]
    # inputs quantised to float32 so that both sides see the same numbers
    q = lambda a: np.asarray(a, np.float32).astype(np.float64)
    ev.hit_xyz, ev.hit_lcov = q(ev.hit_xyz), q(ev.hit_lcov)
    align = q(rng.normal(0, 1e-3, (g.n_layers, 3)))
    x0 = q(g.x0 * (1 + 0.2 * rng.random(g.n_layers)))
    T = hits.shape[0]
    up = dict(g_chi2=q(rng.normal(size=T)), g_par=q(rng.normal(size=(T, 6)) * [1, 1, 1, 10, 1, 1]),
              g_cov=q(rng.normal(size=(T, 21)) * 100))
    return g, ev, hits, q(sp), q(sc), align, x0, up


EPS32 = 2.0 ** -24


def _floors(g, ev, hits, sp, sc, up, align, x0):
    """FP32 floors of the gradient components (module docstring): hits,
    per-layer (dr, dphi, dz) [L, 3] and thickness [L]."""
    import oracle
    used = hits[hits >= 0]
    r_max = float(np.abs(g.table()[:, 1:4]).max())
    var_min = float(ev.hit_lcov[used][:, :2].min())
    f_hit = 8 * EPS32 * r_max / var_min
    n = np.bincount(ev.hit_layer[used], minlength=g.n_layers).astype(np.float64)
    radius = np.where(np.asarray(g.kind) == 0, np.abs(g.table()[:, 1]), np.abs(g.table()[:, 3]))
    f_layer = np.stack([f_hit * np.sqrt(n), f_hit * np.sqrt(n) * radius, f_hit * np.sqrt(n)], 1)
    # sum over tracks of |each track's term|, from the oracle track by track
    geo = oracle.Geo.of(g)
    abs_a, abs_x = np.zeros((g.n_layers, 3)), np.zeros(g.n_layers)
    for t in range(hits.shape[0]):
        pick = lambda k: None if up.get(k) is None else up[k][t:t + 1]
        _, ga, gx = oracle.fit_grad(geo, ev.hit_xyz, ev.hit_lcov, ev.hit_layer, hits[t:t + 1], sp[t:t + 1],
                                    sc[t:t + 1], up["g_chi2"][t:t + 1], g_par=pick("g_par"), g_cov=pick("g_cov"),
                                    align=align, x0=x0)
        abs_a += np.abs(ga)
        abs_x += np.abs(gx)
    return f_hit, np.maximum(f_layer, 1e-4 * abs_a), 1e-4 * abs_x


def _component_errors(got, ref, floor):
    """(largest |g - r| / (1e-3 |r| + floor) over the components, norm-wise
    relative error of the group).  The first must not exceed 1."""
    err = np.abs(got - ref)
    bound = GRAD_RTOL * np.abs(ref) + floor
    ratio = np.where(err > 0, err / np.where(bound > 0, bound, 1e-300), 0.0)
    return float(ratio.max()), float(np.linalg.norm(got - ref) / np.linalg.norm(ref))


@pytest.mark.parametrize("upstream", ["chi2", "all"])
def test_adjoint_matches_oracle_gradient(upstream):
    import oracle
    import paper_2002_06295_gb300 as mkf
    g, ev, hits, sp, sc, align, x0, up = _inputs()
    if upstream == "chi2":
        up = dict(g_chi2=up["g_chi2"], g_par=None, g_cov=None)
    dev = torch.device("cuda", 0)
    ctx = make_ctx(g)
    T, K = hits.shape
    xyz_d, lcov_d, lay_d, hits_d = f32(ev.hit_xyz.T, dev), f32(ev.hit_lcov.T, dev), i32(ev.hit_layer, dev), i32(hits, dev)
    sp_d, sc_d, al_d, x0_d = f32(sp.T, dev), f32(sc.T, dev), f32(align, dev), f32(x0, dev)
    ckpt = torch.empty((K, 27, T), dtype=torch.float32, device=dev)
    mkf.mkf_fit_tracks(ctx, xyz_d, lcov_d, lay_d, hits_d, sp_d, sc_d, align=al_d, x0=x0_d, ckpt=ckpt)
    gd = {k: (None if v is None else f32(v.T if v.ndim == 2 else v, dev)) for k, v in up.items()}
    out = mkf.mkf_fit_tracks_adjoint(ctx, xyz_d, lcov_d, lay_d, hits_d, sp_d, sc_d, ckpt, align=al_d, x0=x0_d, **gd)
    mkf.mkf_sync(ctx)
    gh = out["g_hit"].cpu().numpy().T.astype(np.float64)
    ga = out["g_align"].cpu().numpy().astype(np.float64)
    gx = out["g_x0"].cpu().numpy().astype(np.float64)
    rh, ra, rx = oracle.fit_grad(oracle.Geo.of(g), ev.hit_xyz, ev.hit_lcov, ev.hit_layer, hits, sp, sc, up["g_chi2"],
                                 g_par=up["g_par"], g_cov=up["g_cov"], align=align, x0=x0)
    used = np.unique(hits[hits >= 0])
    f_hit, f_layer, f_x0 = _floors(g, ev, hits, sp, sc, up, align, x0)
    report = {}
    for name, a, b, f in (("hit_x", gh[used, 0], rh[used, 0], f_hit), ("hit_y", gh[used, 1], rh[used, 1], f_hit),
                          ("hit_z", gh[used, 2], rh[used, 2], f_hit), ("align_dr", ga[:, 0], ra[:, 0], f_layer[:, 0]),
                          ("align_dphi", ga[:, 1], ra[:, 1], f_layer[:, 1]),
                          ("align_dz", ga[:, 2], ra[:, 2], f_layer[:, 2]), ("x0", gx, rx, f_x0)):
        report[name] = _component_errors(a, b, f)
    print("adjoint vs oracle (worst component / its bound, norm-wise):", report)
    for name, (worst, enorm) in report.items():
        assert enorm < GRAD_RTOL, (name, report)
        assert worst <= 1.0, (name, report)
    ctx.close()


def test_adjoint_launch_shapes_agree():
    """One thread per track and eight lanes per track compute the same
    per-track adjoint: hit gradients (each hit here belongs to one track) are
    equal bit for bit; layer sums, accumulated by atomics in launch order,
    agree to rounding."""
    import paper_2002_06295_gb300 as mkf
    g, ev, hits, sp, sc, align, x0, up = _inputs(n=500, seed=24)
    dev = torch.device("cuda", 0)
    ctx = make_ctx(g)
    T, K = hits.shape
    xyz_d, lcov_d, lay_d, hits_d = f32(ev.hit_xyz.T, dev), f32(ev.hit_lcov.T, dev), i32(ev.hit_layer, dev), i32(hits, dev)
    sp_d, sc_d, al_d, x0_d = f32(sp.T, dev), f32(sc.T, dev), f32(align, dev), f32(x0, dev)
    ckpt = torch.empty((K, 27, T), dtype=torch.float32, device=dev)
    mkf.mkf_fit_tracks(ctx, xyz_d, lcov_d, lay_d, hits_d, sp_d, sc_d, align=al_d, x0=x0_d, ckpt=ckpt)
    gd = {k: f32(v.T if v.ndim == 2 else v, dev) for k, v in up.items()}
    res = {}
    for lanes in (1, 8):
        mkf.mkf_set_adjoint_config(ctx, lanes)
        out = mkf.mkf_fit_tracks_adjoint(ctx, xyz_d, lcov_d, lay_d, hits_d, sp_d, sc_d, ckpt, align=al_d, x0=x0_d,
                                         **gd)
        mkf.mkf_sync(ctx)
        res[lanes] = {k: v.cpu().numpy().astype(np.float64) for k, v in out.items()}
    assert np.array_equal(res[1]["g_hit"], res[8]["g_hit"])
    for k in ("g_align", "g_x0"):
        a, b = res[1][k], res[8][k]
        assert np.abs(a - b).max() <= 1e-5 * np.abs(a).max(), k
    with pytest.raises(mkf.MkfError):
        mkf.mkf_set_adjoint_config(ctx, 4)
    ctx.close()


def test_adjoint_matches_central_differences():
    """FP64 central differences of the oracle's fit, h = 1e-6, on a few inputs."""
    import oracle
    import paper_2002_06295_gb300 as mkf
    g, ev, hits, sp, sc, align, x0, up = _inputs(n=40, seed=22)
    dev = torch.device("cuda", 0)
    ctx = make_ctx(g)
    T, K = hits.shape
    geo = oracle.Geo.of(g)
    xyz_d, lcov_d, lay_d, hits_d = f32(ev.hit_xyz.T, dev), f32(ev.hit_lcov.T, dev), i32(ev.hit_layer, dev), i32(hits, dev)
    sp_d, sc_d, al_d, x0_d = f32(sp.T, dev), f32(sc.T, dev), f32(align, dev), f32(x0, dev)
    ckpt = torch.empty((K, 27, T), dtype=torch.float32, device=dev)
    mkf.mkf_fit_tracks(ctx, xyz_d, lcov_d, lay_d, hits_d, sp_d, sc_d, align=al_d, x0=x0_d, ckpt=ckpt)
    out = mkf.mkf_fit_tracks_adjoint(ctx, xyz_d, lcov_d, lay_d, hits_d, sp_d, sc_d, ckpt, align=al_d, x0=x0_d,
                                     g_chi2=f32(up["g_chi2"], dev))
    mkf.mkf_sync(ctx)
    gh = out["g_hit"].cpu().numpy().T
    ga = out["g_align"].cpu().numpy()
    gx = out["g_x0"].cpu().numpy()

    def loss(hx=ev.hit_xyz, al=align, xx=x0):
        _, _, chi2, _ = oracle.fit(geo, hx, ev.hit_lcov, ev.hit_layer, hits, sp, sc, align=al, x0=xx)
        return float(up["g_chi2"] @ chi2)

    h = 1e-6
    f_hit, f_layer, f_x0 = _floors(g, ev, hits, sp, sc, dict(g_chi2=up["g_chi2"]), align, x0)
    rng = np.random.default_rng(5)
    for hid in rng.choice(np.unique(hits[hits >= 0]), 8, replace=False):
        for c in range(3):
            a = ev.hit_xyz.copy(); b = a.copy(); a[hid, c] += h; b[hid, c] -= h
            fd = (loss(hx=a) - loss(hx=b)) / (2 * h)
            assert abs(gh[hid, c] - fd) <= GRAD_RTOL * abs(fd) + f_hit, (hid, c, gh[hid, c], fd)
    for l in (0, 6, 13):
        for c in range(3):
            a = align.copy(); b = align.copy(); a[l, c] += h; b[l, c] -= h
            fd = (loss(al=a) - loss(al=b)) / (2 * h)
            assert abs(ga[l, c] - fd) <= GRAD_RTOL * abs(fd) + f_layer[l, c], (l, c, ga[l, c], fd)
        # thickness: x/X0 ~ 0.01 enters through the scattering variance only,
        # so its central difference takes a 1e-4 step (five-point stencil)
        hx = 1e-4

        def at(k):
            a = x0.copy()
            a[l] += k * hx
            return loss(xx=a)
        fd = (-at(2) + 8 * at(1) - 8 * at(-1) + at(-2)) / (12 * hx)
        assert abs(gx[l] - fd) <= GRAD_RTOL * abs(fd) + f_x0[l], (l, gx[l], fd, f_x0[l])
    ctx.close()


def test_autograd_function():
    """torch.autograd through the C ABI: the gradient of a scalar loss equals
    the direct adjoint call; inputs without requires_grad get no gradient."""
    import paper_2002_06295_gb300 as mkf
    from paper_2002_06295_gb300.autograd import kalman_fit
    g, ev, hits, sp, sc, align, x0, up = _inputs(n=200, seed=23)
    dev = torch.device("cuda", 0)
    ctx = make_ctx(g)
    xyz = f32(ev.hit_xyz.T, dev).requires_grad_(True)
    al = f32(align, dev).requires_grad_(True)
    xx = f32(x0, dev).requires_grad_(True)
    lcov, lay, hd = f32(ev.hit_lcov.T, dev), i32(ev.hit_layer, dev), i32(hits, dev)
    chi2, par, cov, ok = kalman_fit(ctx, xyz, lcov, lay, hd, f32(sp.T, dev), f32(sc.T, dev), align=al, x0=xx)
    w = f32(up["g_chi2"], dev)
    (w * chi2).sum().add(par[3].sum()).backward()
    T, K = hits.shape
    ckpt = torch.empty((K, 27, T), dtype=torch.float32, device=dev)
    mkf.mkf_fit_tracks(ctx, xyz.detach(), lcov, lay, hd, f32(sp.T, dev), f32(sc.T, dev), align=al.detach(),
                       x0=xx.detach(), ckpt=ckpt)
    gp = torch.zeros((6, T), dtype=torch.float32, device=dev)
    gp[3] = 1
    ref = mkf.mkf_fit_tracks_adjoint(ctx, xyz.detach(), lcov, lay, hd, f32(sp.T, dev), f32(sc.T, dev), ckpt,
                                     g_chi2=w, g_par=gp, align=al.detach(), x0=xx.detach())
    mkf.mkf_sync(ctx)
    assert torch.allclose(xyz.grad, ref["g_hit"], rtol=1e-6, atol=0)
    assert torch.allclose(al.grad, ref["g_align"], rtol=1e-4, atol=1e-6 * float(ref["g_align"].abs().max()))
    assert torch.allclose(xx.grad, ref["g_x0"], rtol=1e-4, atol=1e-6 * float(ref["g_x0"].abs().max()))
    ctx.close()


def test_fit_gradient_full_size_sampled_tracks():
    """C4 at full size (100k tracks x 14 hits, barrel of 14 cylinders) in one
    launch as the bench times it.  Each hit belongs to one track, so the
    gradient of sum chi2 with respect to a sampled track's hits is that track's
    alone: it is compared, with the track's chi2, against the oracle's
    dual-number gradient of that track."""
    import oracle
    import paper_2002_06295_gb300 as mkf
    g = synth.geometry_barrel14()
    rng = np.random.default_rng(synth.config_seed(4))
    ev = synth.simulate_event(g, 100000, rng, pt_range=(1.0, 10.0), eta_max=0.8)
    keep = (ev.true_hits >= 0).sum(1) == 14
    hits, sp, sc = ev.true_hits[keep], ev.seed_par[keep], ev.seed_cov[keep]
    q = lambda a: np.asarray(a, np.float32).astype(np.float64)
    ev.hit_xyz, ev.hit_lcov = q(ev.hit_xyz), q(ev.hit_lcov)
    sp, sc = q(sp), q(sc)
    T, K = hits.shape
    assert T > 50000
    dev = torch.device("cuda", 0)
    ctx = make_ctx(g)
    xyz_d, lcov_d, lay_d, hits_d = f32(ev.hit_xyz.T, dev), f32(ev.hit_lcov.T, dev), i32(ev.hit_layer, dev), i32(hits, dev)
    ckpt = torch.empty((K, 27, T), dtype=torch.float32, device=dev)
    fo = mkf.mkf_fit_tracks(ctx, xyz_d, lcov_d, lay_d, hits_d, f32(sp.T, dev), f32(sc.T, dev), ckpt=ckpt)
    out = mkf.mkf_fit_tracks_adjoint(ctx, xyz_d, lcov_d, lay_d, hits_d, f32(sp.T, dev), f32(sc.T, dev), ckpt,
                                     g_chi2=torch.ones(T, dtype=torch.float32, device=dev))
    mkf.mkf_sync(ctx)
    gh = out["g_hit"].cpu().numpy().T.astype(np.float64)
    chi2 = fo["chi2"].cpu().numpy().astype(np.float64)
    sel = np.random.default_rng(25).choice(T, 60, replace=False)
    geo = oracle.Geo.of(g)
    rh, _, _ = oracle.fit_grad(geo, ev.hit_xyz, ev.hit_lcov, ev.hit_layer, hits[sel], sp[sel], sc[sel], np.ones(sel.size))
    _, _, rchi2, _ = oracle.fit(geo, ev.hit_xyz, ev.hit_lcov, ev.hit_layer, hits[sel], sp[sel], sc[sel])
    # each sampled track's chi2 on its own
    assert np.all(np.abs(chi2[sel] - rchi2) <= 1e-3 * rchi2), np.max(np.abs(chi2[sel] - rchi2) / rchi2)
    used = hits[sel].ravel()
    f_hit = 8 * EPS32 * float(np.abs(g.table()[:, 1:4]).max()) / float(ev.hit_lcov[used][:, :2].min())
    for c in range(3):
        worst, enorm = _component_errors(gh[used, c], rh[used, c], f_hit)
        assert enorm < GRAD_RTOL and worst <= 1.0, (c, worst, enorm)
    ctx.close()


def test_adjoint_on_tracks_built_on_the_cmslike_event():
    """Tracks built on the C2 event, as the bench's step fits them.  A slow
    particle near theta = pi/2 can drift from one endcap disk to the next over
    several turns of its helix; there the fit's reverse sweep is not accurate
    in FP32, so the forward fit reports such tracks with ok = 2 and the
    adjoint leaves them out.  Checked here: ok = 2 marks exactly the tracks
    with a transport onto a disk of one turn or more (recomputed in FP64 from
    the checkpoints); the adjoint of those tracks alone is zero; the gradients
    of the whole event are finite; and on a sample of the other tracks they
    match the oracle's dual-number gradient at this module's bar."""
    import oracle
    import paper_2002_06295_gb300 as mkf
    from _util import gpu_build
    ev = synth.make_config_event(2)
    q = lambda a: np.asarray(a, np.float32).astype(np.float64)
    ev.hit_xyz, ev.hit_lcov = q(ev.hit_xyz), q(ev.hit_lcov)
    g = ev.geom
    ctx = make_ctx(g)
    b = gpu_build(ctx, [ev], max_cands=6)
    keep = (b["hits"] >= 0).sum(1) >= 4
    hits, sp, sc = b["hits"][keep], q(ev.seed_par[keep]), q(ev.seed_cov[keep])
    T, K = hits.shape
    dev = torch.device("cuda", 0)
    xyz_d, lcov_d, lay_d = f32(ev.hit_xyz.T, dev), f32(ev.hit_lcov.T, dev), i32(ev.hit_layer, dev)

    def fit_and_adjoint(sel):
        hd, spd, scd = i32(hits[sel], dev), f32(sp[sel].T, dev), f32(sc[sel].T, dev)
        ckpt = torch.empty((K, 27, len(sel)), dtype=torch.float32, device=dev)
        fo = mkf.mkf_fit_tracks(ctx, xyz_d, lcov_d, lay_d, hd, spd, scd, ckpt=ckpt)
        go = mkf.mkf_fit_tracks_adjoint(ctx, xyz_d, lcov_d, lay_d, hd, spd, scd, ckpt,
                                        g_chi2=torch.ones(len(sel), dtype=torch.float32, device=dev))
        mkf.mkf_sync(ctx)
        return (fo["ok"].cpu().numpy(), ckpt.cpu().numpy().astype(np.float64),
                {k: v.cpu().numpy().astype(np.float64) for k, v in go.items()})

    ok, ck, gall = fit_and_adjoint(np.arange(T))
    for k, v in gall.items():
        assert np.isfinite(v).all(), k
    # the rule, in FP64 from the same checkpointed states: s = (z_disk - z) tan(theta)
    tab = np.asarray(g.table())
    kind = np.asarray(g.kind)
    c_kappa = -synth.events.ALPHA * g.bz
    turns = np.zeros(T)
    for t in range(T):
        for k in range(K):
            h = hits[t, k]
            if h < 0 or kind[ev.hit_layer[h]] != 1:
                continue
            p = ck[k, :6, t]
            if not np.isfinite(p[0]):
                break
            s = (tab[ev.hit_layer[h], 1] - p[2]) * np.tan(p[5])
            if s > 0:
                turns[t] = max(turns[t], abs(s * c_kappa * p[3]) / (2 * np.pi))
    clear = np.abs(turns - 1.0) > 1e-4
    print("built C2 tracks: %d, ok=2: %d, ok=0: %d" % (T, (ok == 2).sum(), (ok == 0).sum()))
    assert np.array_equal((ok == 2)[clear], (turns >= 1.0)[clear])
    assert (ok == 2).sum() > 20 and (ok == 0).mean() < 0.02
    # those tracks alone: nothing
    _, _, g2 = fit_and_adjoint(np.where(ok == 2)[0])
    for k, v in g2.items():
        assert not v.any(), k
    # a sample of the others against the oracle
    rng = np.random.default_rng(26)
    cand = rng.choice(np.where(ok == 1)[0], 260, replace=False)
    geo = oracle.Geo.of(g)
    _, _, _, fok = oracle.fit(geo, ev.hit_xyz, ev.hit_lcov, ev.hit_layer, hits[cand], sp[cand], sc[cand])
    sel = cand[fok.astype(bool)][:200]
    _, _, gs = fit_and_adjoint(sel)
    ones = np.ones(sel.size)
    rh, ra, rx = oracle.fit_grad(geo, ev.hit_xyz, ev.hit_lcov, ev.hit_layer, hits[sel], sp[sel], sc[sel], ones)
    f_hit, f_layer, f_x0 = _floors(g, ev, hits[sel], sp[sel], sc[sel], dict(g_chi2=ones), None, None)
    used = np.unique(hits[sel][hits[sel] >= 0])
    gh = gs["g_hit"].T
    report = {}
    for name, a, r, f in (("hit_x", gh[used, 0], rh[used, 0], f_hit), ("hit_y", gh[used, 1], rh[used, 1], f_hit),
                          ("hit_z", gh[used, 2], rh[used, 2], f_hit),
                          ("align_dr", gs["g_align"][:, 0], ra[:, 0], f_layer[:, 0]),
                          ("align_dphi", gs["g_align"][:, 1], ra[:, 1], f_layer[:, 1]),
                          ("align_dz", gs["g_align"][:, 2], ra[:, 2], f_layer[:, 2]), ("x0", gs["g_x0"], rx, f_x0)):
        report[name] = _component_errors(a, r, f)
    print("built C2 tracks, adjoint vs oracle (worst component / its bound, norm-wise):", report)
    for name, (worst, enorm) in report.items():
        assert enorm < GRAD_RTOL, (name, report)
        assert worst <= 1.0, (name, report)
    ctx.close()
