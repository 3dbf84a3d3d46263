"""Pins of the overlap-hit oracle (Sec. 3: hits in overlapping modules, more
than one hit per layer assigned to a track) against facts that do not come
from its selection code:
  * an exact copy of a track hit is chosen as that crossing's overlap hit, with
    the chi2 of a measurement equal to the first one against the fitted state
    after it (computed here in numpy from the fit oracle's state);
  * hits on other layers, in other events, on the far side of the axis, or
    the track's own hit are never chosen; of two identical copies the smaller
    id is; the chi2 cut is strict; a candidate just outside the
    adjacent-module box is not taken, one just inside is;
  * on simulated events with overlapping modules, the simulation's own overlap
    hits are found for more than 95 % of the crossings that have one, and
    fewer than 5 % of the crossings without one get a hit."""
import numpy as np

import oracle
import synth.events as sev


def _tracks(ev, n):
    """First n tracks with >= 6 hits: hit lists in crossing order, seeds."""
    rows, par, cov = [], [], []
    for t in range(ev.n_seeds):
        h = ev.true_hits[t]
        if (h >= 0).sum() >= 6:
            rows.append(h)
            par.append(ev.seed_par[t])
            cov.append(ev.seed_cov[t])
        if len(rows) == n:
            break
    return np.array(rows, np.int32), np.array(par), np.array(cov)


def _chi2_dup(geo, ev, hits_t, k, par, cov):
    """chi2 of a copy of hit k against the fit oracle's state after hit k."""
    sub = hits_t.copy()
    sub[k + 1:] = -1
    p, C, _, ok = oracle.fit(geo, ev.hit_xyz, ev.hit_lcov, ev.hit_layer, sub[None], par[None], cov[None])
    assert ok[0]
    p, C = p[0], oracle.unpack_cov(C[0])
    h = hits_t[k]
    x, y, z = ev.hit_xyz[h]
    ph = np.arctan2(y, x)
    c, s = np.cos(ph), np.sin(ph)
    Hm = np.zeros((2, 6))
    Hm[0, 0], Hm[0, 1] = -s, c
    if ev.geom.kind[ev.hit_layer[h]] == 0:
        Hm[1, 2] = 1.0
        w = z
    else:
        Hm[1, 0], Hm[1, 1] = c, s
        w = np.hypot(x, y)
    r = np.array([0.0, w]) - Hm @ p
    va, vb, vab = ev.hit_lcov[h]
    R = np.array([[va, vab], [vab, vb]]) + Hm @ C @ Hm.T
    return float(r @ np.linalg.solve(R, r))


def test_exact_copy_is_the_overlap_with_its_closed_form_chi2():
    ev = sev.make_config_event(1, n_tracks=60)      # barrel, no noise
    geo = oracle.Geo.of(ev.geom)
    hits, par, cov = _tracks(ev, 5)
    t, k = 2, 4
    h = hits[t, k]
    xyz = np.concatenate([ev.hit_xyz, ev.hit_xyz[h:h + 1]])
    lcov = np.concatenate([ev.hit_lcov, ev.hit_lcov[h:h + 1]])
    lay = np.concatenate([ev.hit_layer, ev.hit_layer[h:h + 1]])
    r = oracle.overlaps(geo, xyz, lcov, lay, hits, par, cov, chi2_cut=1e9)
    H = ev.n_hits
    assert r["hit"][t, k] == H
    ref = _chi2_dup(geo, ev, hits[t], k, par[t], cov[t])
    assert abs(r["chi2"][t, k] - ref) <= 1e-9 * max(1.0, ref)
    # the cut is strict
    r2 = oracle.overlaps(geo, xyz, lcov, lay, hits, par, cov, chi2_cut=ref * (1 - 1e-9))
    assert r2["hit"][t, k] != H
    # two identical copies: the smaller id
    xyz3 = np.concatenate([xyz, ev.hit_xyz[h:h + 1]])
    lcov3 = np.concatenate([lcov, ev.hit_lcov[h:h + 1]])
    lay3 = np.concatenate([lay, ev.hit_layer[h:h + 1]])
    r3 = oracle.overlaps(geo, xyz3, lcov3, lay3, hits, par, cov, chi2_cut=1e9)
    assert r3["hit"][t, k] == H and r3["gap"][t, k] == 0.0


def test_never_other_layers_events_far_side_or_itself():
    ev = sev.make_config_event(1, n_tracks=60)
    geo = oracle.Geo.of(ev.geom)
    hits, par, cov = _tracks(ev, 5)
    t, k = 1, 3
    h = hits[t, k]
    other = (ev.hit_layer[h] + 1) % ev.geom.n_layers
    mirror = ev.hit_xyz[h] * np.array([-1.0, -1.0, 1.0])
    xyz = np.concatenate([ev.hit_xyz, ev.hit_xyz[h:h + 1], mirror[None]])
    lcov = np.concatenate([ev.hit_lcov, ev.hit_lcov[h:h + 1], ev.hit_lcov[h:h + 1]])
    lay = np.concatenate([ev.hit_layer, [other, ev.hit_layer[h]]]).astype(np.int32)
    r = oracle.overlaps(geo, xyz, lcov, lay, hits, par, cov, chi2_cut=1e9)
    H = ev.n_hits
    assert r["hit"][t, k] not in (H, H + 1, h)
    # a copy in a second event is not a candidate for the first
    xyz2 = np.concatenate([ev.hit_xyz, ev.hit_xyz[h:h + 1]])
    lcov2 = np.concatenate([ev.hit_lcov, ev.hit_lcov[h:h + 1]])
    lay2 = np.concatenate([ev.hit_layer, ev.hit_layer[h:h + 1]])
    r2 = oracle.overlaps(geo, xyz2, lcov2, lay2, hits, par, cov, ev_hit_off=np.array([0, H, H + 1]), chi2_cut=1e9)
    assert r2["hit"][t, k] != H
    # with every other hit of the layer gone, nothing is found
    keep = np.nonzero((ev.hit_layer != ev.hit_layer[h]) | (np.arange(H) == h))[0]
    remap = -np.ones(H, np.int32)
    remap[keep] = np.arange(keep.size)
    hk = np.where(hits >= 0, remap[np.maximum(hits, 0)], -1)
    hk = np.where((hits >= 0) & (hk < 0), -1, hk)
    r3 = oracle.overlaps(geo, ev.hit_xyz[keep], ev.hit_lcov[keep], ev.hit_layer[keep], hk, par, cov, chi2_cut=1e9)
    assert r3["hit"][t, k] == -1 and np.isinf(r3["best"][t, k])


def test_adjacent_module_box():
    """With hit variances so large that chi2 cannot decide, the box does: a
    copy of the hit turned by just under max_drphi / R about the axis is taken,
    just over is not; the same in z with max_dw."""
    ev = sev.make_config_event(1, n_tracks=60)
    geo = oracle.Geo.of(ev.geom)
    hits, par, cov = _tracks(ev, 3)
    t, k = 0, 3
    h = hits[t, k]
    R = ev.geom.pos[ev.hit_layer[h]]
    lcov = ev.hit_lcov.copy()
    lcov[:, 0] = lcov[:, 1] = 100.0   # 10 cm resolution: every nearby hit has a tiny chi2
    H = ev.n_hits
    for f, taken in ((0.99, True), (1.01, False)):
        d = f * 1.0 / R
        x, y, z = ev.hit_xyz[h]
        c = np.array([[x * np.cos(d) - y * np.sin(d), x * np.sin(d) + y * np.cos(d), z]])
        r = oracle.overlaps(geo, np.concatenate([ev.hit_xyz, c]), np.concatenate([lcov, lcov[h:h + 1]]),
                            np.concatenate([ev.hit_layer, ev.hit_layer[h:h + 1]]), hits, par, cov, chi2_cut=1e9,
                            max_drphi=1.0, max_dw=10.0)
        assert (r["hit"][t, k] == H) == taken, f
    for dz, taken in ((9.9, True), (10.1, False)):
        c = ev.hit_xyz[h:h + 1] + np.array([[0.0, 0.0, dz]])
        r = oracle.overlaps(geo, np.concatenate([ev.hit_xyz, c]), np.concatenate([lcov, lcov[h:h + 1]]),
                            np.concatenate([ev.hit_layer, ev.hit_layer[h:h + 1]]), hits, par, cov, chi2_cut=1e9,
                            max_drphi=1.0, max_dw=10.0)
        assert (r["hit"][t, k] == H) == taken, dz


def test_simulated_overlaps_are_recovered():
    ev = sev.make_config_event(2, n_tracks=800, overlap_frac=0.3)
    geo = oracle.Geo.of(ev.geom)
    T = ev.n_seeds
    sel = [t for t in range(T) if (ev.true_hits[t] >= 0).sum() >= 8]
    hits = ev.true_hits[sel].astype(np.int32)
    r = oracle.overlaps(geo, ev.hit_xyz, ev.hit_lcov, ev.hit_layer, hits, ev.seed_par[sel], ev.seed_cov[sel],
                        chi2_cut=20.0)
    truth = ev.true_overlap[sel]
    has = (truth >= 0) & (hits >= 0)
    # skip the first three hits of each track (the fitted state is still loose there)
    early = np.zeros_like(has)
    for i, row in enumerate(hits):
        idx = np.nonzero(row >= 0)[0][:3]
        early[i, idx] = True
    a = has & ~early
    b = ~has & (hits >= 0) & ~early
    assert a.sum() > 300
    found = (r["hit"][a] == truth[a]).mean()
    fake = (r["hit"][b] >= 0).mean()
    assert found > 0.95, found
    assert fake < 0.05, fake
