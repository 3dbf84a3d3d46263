"""Seeded simulation of synthetic events shaped like the paper's workloads.

Truth simulation (physics, not reconstruction): prompt charged particles start
at the origin and move on helices in the uniform solenoid field.  Each particle
crosses the layers outward in order of transverse path length; every crossing
inside a layer's acceptance leaves one hit, smeared inside the surface, and
applies a multiple-scattering kick to the direction (Highland width, pion mass,
no energy loss, q/pT held fixed).  A particle stops when no further layer is
reachable.  Noise hits are spread over the layers in proportion to the signal
hits, uniform in (phi, z) on a barrel and uniform in area on a disk.  Seeds are
the true vertex parameters smeared by 5 %.

Random draws: numpy ``default_rng((20020 + config) * 1000 + event)``.

Units: cm, GeV, tesla, radians.  Parameter vector (x, y, z, kappa = q/pT,
phi = momentum azimuth, theta = polar angle).
"""
from dataclasses import dataclass

import numpy as np

from .geometry import (KIND_BARREL, Geometry, geometry_barrel10, geometry_barrel14,
                       geometry_cmslike)

ALPHA = 0.00299792458      # GeV / (T cm): curvature constant of a unit charge
PION_MASS = 0.13957        # GeV
NAV_EPS = 1e-6             # cm: a surface must lie strictly beyond the reference radius / |z|


def config_seed(config: int, event: int = 0) -> int:
    return (20020 + config) * 1000 + event


@dataclass
class Event:
    geom: Geometry
    hit_xyz: np.ndarray       # [H, 3] float64 global positions
    hit_lcov: np.ndarray      # [H, 3] float64 local covariance (var_a, var_b, cov_ab)
    hit_layer: np.ndarray     # [H] int32
    hit_track: np.ndarray     # [H] int32, truth particle id, -1 for noise
    seed_par: np.ndarray      # [S, 6] float64
    seed_cov: np.ndarray      # [S, 21] float64, packed lower triangle (row-major)
    true_par: np.ndarray      # [S, 6] float64 true vertex parameters
    true_hits: np.ndarray     # [S, L] int32 hit ids in crossing order, -1 padded
    true_layers: np.ndarray   # [S, L] int32 crossed layer ids, -1 padded
    true_state: np.ndarray = None   # [S, L, 6] at each crossing: position, kappa, direction after the kick
    true_overlap: np.ndarray = None   # [S, L] int32 second hit of each crossing (overlapping module), -1 if none

    @property
    def n_hits(self):
        return int(self.hit_layer.shape[0])

    @property
    def n_seeds(self):
        return int(self.seed_par.shape[0])


@dataclass
class EventBatch:
    """Several events concatenated, with CSR offsets (hits and seeds)."""
    geom: Geometry
    events: list
    hit_off: np.ndarray       # [E+1] int64
    seed_off: np.ndarray      # [E+1] int64

    def cat(self, name):
        return np.concatenate([getattr(e, name) for e in self.events], 0)

    @property
    def n_events(self):
        return len(self.events)


def cov_index(i, j):
    if i < j:
        i, j = j, i
    return i * (i + 1) // 2 + j


def _sinc(u):
    return np.sinc(u / np.pi)


def _position_at(x, y, z, phi, cot, omega, s):
    u = 0.5 * omega * s
    f = s * _sinc(u)
    return x + f * np.cos(phi + u), y + f * np.sin(phi + u), z + s * cot


def _cylinder_path(x, y, phi, omega, r):
    """Smallest positive transverse path to the circle x^2 + y^2 = r^2, inf if
    the particle's circle does not reach it (circle-circle intersection)."""
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / omega
        cx = x - np.sin(phi) * inv
        cy = y + np.cos(phi) * inv
        R = np.abs(inv)
        d = np.hypot(cx, cy)
        ok = (d <= r + R) & (d >= np.abs(r - R)) & (d > 0)
        a = (r * r - R * R + d * d) / (2 * d)
        h = np.sqrt(np.maximum(r * r - a * a, 0.0))
        ux, uy = cx / d, cy / d
        best = np.full(x.shape, np.inf)
        for sgn in (1.0, -1.0):
            qx = a * ux - sgn * h * uy
            qy = a * uy + sgn * h * ux
            v0x, v0y = x - cx, y - cy
            v1x, v1y = qx - cx, qy - cy
            ang = np.arctan2(v0x * v1y - v0y * v1x, v0x * v1x + v0y * v1y) * np.sign(omega)
            ang = np.where(ang <= 1e-12, ang + 2 * np.pi, ang)
            s = ang * R
            best = np.where(ok & (s < best), s, best)
    return best


def tracking_radius(geom):
    """Outer radius of the tracking volume: the largest barrel radius or disk
    outer edge."""
    return float(max(np.max(np.where(geom.kind == KIND_BARREL, geom.pos, geom.hi)), 0.0))


def _highland(t_eff, kappa, theta):
    p = 1.0 / (np.abs(kappa) * np.sin(theta))
    beta_p = p * p / np.sqrt(p * p + PION_MASS ** 2)
    return 0.0136 / beta_p * np.sqrt(t_eff) * (1.0 + 0.038 * np.log(t_eff))


def simulate_event(geom: Geometry, n_tracks: int, rng: np.random.Generator, *,
                   pt_range=(0.5, 10.0), pt_log=False, eta_max=1.0, noise_frac=0.0,
                   seed_smear=0.05, kick=True, overlap_frac=0.0):
    """overlap_frac: probability that a barrel crossing also leaves a second,
    independently smeared hit on the same layer (a stand-in for the track
    passing through two overlapping modules; the collapsed layer puts both on
    its radius).  With 0 no extra random numbers are drawn."""
    L = geom.n_layers
    T = n_tracks
    r_max = tracking_radius(geom)
    if pt_log:
        pt = np.exp(rng.uniform(np.log(pt_range[0]), np.log(pt_range[1]), T))
    else:
        pt = rng.uniform(pt_range[0], pt_range[1], T)
    eta = rng.uniform(-eta_max, eta_max, T)
    phi0 = rng.uniform(-np.pi, np.pi, T)
    q = np.where(rng.random(T) < 0.5, -1.0, 1.0)
    theta0 = 2.0 * np.arctan(np.exp(-eta))
    kappa = q / pt
    true_par = np.stack([np.zeros(T), np.zeros(T), np.zeros(T), kappa, phi0, theta0], 1)

    x = np.zeros(T); y = np.zeros(T); z = np.zeros(T)
    phi = phi0.copy(); theta = theta0.copy()
    omega = -ALPHA * geom.bz * kappa
    rho_ref = np.zeros(T); zeta_ref = np.zeros(T)
    alive = np.ones(T, bool)

    hx, hy, hz, hl, ht, ha, hb = [], [], [], [], [], [], []
    cross_layer = np.full((T, L), -1, np.int32)
    cross_hit = np.full((T, L), -1, np.int64)     # provisional index into the signal list
    cross_state = np.full((T, L, 6), np.nan)
    cross_over = np.full((T, L), -1, np.int64)    # provisional index into the overlap list
    ox, oy, oz, ol, ot, oa, ob = [], [], [], [], [], [], []
    n_over = 0
    n_cross = np.zeros(T, np.int64)
    n_sig = 0
    for _ in range(L):
        if not alive.any():
            break
        idx = np.nonzero(alive)[0]
        xs, ys, zs, ps, ts, om = x[idx], y[idx], z[idx], phi[idx], theta[idx], omega[idx]
        cot = np.cos(ts) / np.sin(ts)
        s_exit = _cylinder_path(xs, ys, ps, om, r_max)
        S = np.full((idx.size, L), np.inf)
        for l in range(L):
            if geom.kind[l] == KIND_BARREL:
                r = geom.pos[l]
                cand = r > rho_ref[idx] + NAV_EPS
                s = np.where(cand, _cylinder_path(xs, ys, ps, om, r), np.inf)
                fin = np.isfinite(s)
                zc = np.where(fin, zs + np.where(fin, s, 0) * cot, np.nan)
                acc = fin & (zc >= geom.lo[l]) & (zc <= geom.hi[l])
            else:
                zl = geom.pos[l]
                cand = (np.abs(zl) > zeta_ref[idx] + NAV_EPS) & (np.sign(zl) == np.sign(cot))
                with np.errstate(divide="ignore", invalid="ignore"):
                    s = np.where(cand, (zl - zs) / cot, np.inf)
                s = np.where(s > 0, s, np.inf)
                # a particle that leaves the tracking volume (r > r_max) is lost:
                # the disk must be crossed before the exit
                s = np.where(s < s_exit, s, np.inf)
                fin = np.isfinite(s)
                sx = np.where(fin, s, 0.0)
                px, py, _ = _position_at(xs, ys, zs, ps, cot, om, sx)
                rc = np.hypot(px, py)
                acc = fin & (rc >= geom.lo[l]) & (rc <= geom.hi[l])
            S[:, l] = np.where(acc, s, np.inf)
        nxt = np.argmin(S, 1)
        sbest = S[np.arange(idx.size), nxt]
        stop = ~np.isfinite(sbest)
        alive[idx[stop]] = False
        go = ~stop
        idx, nxt, sbest = idx[go], nxt[go], sbest[go]
        if idx.size == 0:
            break
        xs, ys, zs, ps, ts, om = x[idx], y[idx], z[idx], phi[idx], theta[idx], omega[idx]
        cot = np.cos(ts) / np.sin(ts)
        nx, ny, nz = _position_at(xs, ys, zs, ps, cot, om, sbest)
        nphi = ps + om * sbest
        x[idx], y[idx], z[idx] = nx, ny, nz
        phi[idx] = nphi
        kind = geom.kind[nxt]
        barrel = kind == KIND_BARREL
        rc = np.hypot(nx, ny)
        rho_ref[idx] = np.where(barrel, geom.pos[nxt], np.maximum(rho_ref[idx], rc))
        zeta_ref[idx] = np.where(barrel, np.maximum(zeta_ref[idx], np.abs(nz)), np.abs(geom.pos[nxt]))
        # hit on the nominal surface, smeared inside it
        ga = rng.standard_normal(idx.size)
        gb = rng.standard_normal(idx.size)
        sa = geom.sig_a[nxt]; sb = geom.sig_b[nxt]
        phic = np.arctan2(ny, nx)
        r_on = np.where(barrel, geom.pos[nxt], rc)
        phih = phic + ga * sa / r_on
        rh = np.where(barrel, geom.pos[nxt], rc + gb * sb)
        zh = np.where(barrel, nz + gb * sb, geom.pos[nxt])
        hx.append(rh * np.cos(phih)); hy.append(rh * np.sin(phih)); hz.append(zh)
        hl.append(nxt.astype(np.int32)); ht.append(idx.astype(np.int32))
        ha.append(sa * sa); hb.append(sb * sb)
        k = n_cross[idx]
        cross_layer[idx, k] = nxt
        cross_hit[idx, k] = n_sig + np.arange(idx.size)
        n_cross[idx] += 1
        n_sig += idx.size
        if overlap_frac > 0.0:   # a second hit from an overlapping module
            sel = barrel & (rng.random(idx.size) < overlap_frac)
            ns = int(sel.sum())
            if ns:
                ga2 = rng.standard_normal(ns)
                gb2 = rng.standard_normal(ns)
                r2 = geom.pos[nxt[sel]]
                ph2 = phic[sel] + ga2 * sa[sel] / r2
                ox.append(r2 * np.cos(ph2)); oy.append(r2 * np.sin(ph2)); oz.append(nz[sel] + gb2 * sb[sel])
                ol.append(nxt[sel].astype(np.int32)); ot.append(idx[sel].astype(np.int32))
                oa.append(sa[sel] ** 2); ob.append(sb[sel] ** 2)
                cross_over[idx[sel], k[sel]] = n_over + np.arange(ns)
                n_over += ns
        # multiple-scattering kick after the crossing
        if kick:
            cosinc = np.where(barrel, np.sin(ts) * (nx * np.cos(nphi) + ny * np.sin(nphi)) / rc,
                              np.cos(ts))
            teff = geom.x0[nxt] / np.abs(cosinc)
            th0 = _highland(teff, kappa[idx], ts)
            g1 = rng.standard_normal(idx.size)
            g2 = rng.standard_normal(idx.size)
            phi[idx] = nphi + th0 * g1 / np.sin(ts)
            theta[idx] = np.clip(ts + th0 * g2, 1e-3, np.pi - 1e-3)
        cross_state[idx, k] = np.stack([nx, ny, nz, kappa[idx], phi[idx], theta[idx]], 1)

    if n_sig:
        sx = np.concatenate(hx + ox); sy = np.concatenate(hy + oy); sz = np.concatenate(hz + oz)
        sl = np.concatenate(hl + ol); st = np.concatenate(ht + ot)
        sva = np.concatenate(ha + oa); svb = np.concatenate(hb + ob)
    else:
        sx = sy = sz = sva = svb = np.zeros(0)
        sl = st = np.zeros(0, np.int32)

    # noise hits, per layer in proportion to the signal hits there
    n_noise = int(round(noise_frac * n_sig))
    if n_noise > 0:
        per_layer = np.bincount(sl, minlength=L).astype(np.float64)
        if per_layer.sum() == 0:
            per_layer[:] = 1.0
        nl = rng.choice(L, size=n_noise, p=per_layer / per_layer.sum()).astype(np.int32)
        u1 = rng.random(n_noise); u2 = rng.random(n_noise)
        barrel = geom.kind[nl] == KIND_BARREL
        lo, hi = geom.lo[nl], geom.hi[nl]
        nphi = -np.pi + 2 * np.pi * u1
        r_n = np.where(barrel, geom.pos[nl], np.sqrt(lo * lo + (hi * hi - lo * lo) * u2))
        z_n = np.where(barrel, lo + (hi - lo) * u2, geom.pos[nl])
        sx = np.concatenate([sx, r_n * np.cos(nphi)])
        sy = np.concatenate([sy, r_n * np.sin(nphi)])
        sz = np.concatenate([sz, z_n])
        sl = np.concatenate([sl, nl])
        st = np.concatenate([st, np.full(n_noise, -1, np.int32)])
        sva = np.concatenate([sva, geom.sig_a[nl] ** 2])
        svb = np.concatenate([svb, geom.sig_b[nl] ** 2])

    H = sx.size
    perm = rng.permutation(H)            # new id -> old id
    inv = np.empty(H, np.int64)
    inv[perm] = np.arange(H)
    hit_xyz = np.stack([sx, sy, sz], 1)[perm]
    hit_lcov = np.stack([sva, svb, np.zeros(H)], 1)[perm]
    hit_layer = sl[perm].astype(np.int32)
    hit_track = st[perm].astype(np.int32)
    true_hits = np.where(cross_hit >= 0, inv[np.maximum(cross_hit, 0)], -1).astype(np.int32)
    true_overlap = np.where(cross_over >= 0, inv[np.maximum(n_sig + cross_over, 0)], -1).astype(np.int32)

    # seeds: true vertex parameters smeared by 5 %
    ks = kappa * (1.0 + seed_smear * rng.standard_normal(T))
    ps = phi0 + seed_smear * rng.standard_normal(T)
    ts = np.clip(theta0 + seed_smear * rng.standard_normal(T), 1e-3, np.pi - 1e-3)
    seed_par = np.stack([np.zeros(T), np.zeros(T), np.zeros(T), ks, ps, ts], 1)
    seed_cov = np.zeros((T, 21))
    diag = [0.1 ** 2, 0.1 ** 2, 0.1 ** 2, None, seed_smear ** 2, seed_smear ** 2]
    for i in range(6):
        seed_cov[:, cov_index(i, i)] = (seed_smear * ks) ** 2 if i == 3 else diag[i]
    return Event(geom=geom, hit_xyz=hit_xyz, hit_lcov=hit_lcov, hit_layer=hit_layer,
                 hit_track=hit_track, seed_par=seed_par, seed_cov=seed_cov, true_par=true_par,
                 true_hits=true_hits, true_layers=cross_layer, true_state=cross_state, true_overlap=true_overlap)


# ---------------------------------------------------------------------------
# The five workloads (C1..C5).  Each entry: geometry factory, track count(s),
# kinematic ranges, noise fraction and the reconstruction limits.
WORKLOAD_SPECS = {
    1: dict(name="C1 plain build, barrel10, 100 tracks", geom=geometry_barrel10, n_events=1,
            tracks=100, pt_range=(0.5, 10.0), pt_log=False, eta_max=1.0, noise_frac=0.0,
            chi2_cut=30.0, max_cands=4, max_holes=3, min_hits=4, dup_frac=0.5),
    2: dict(name="C2 plain build, CMS-like 38 surfaces, 5000 tracks", geom=geometry_cmslike,
            n_events=1, tracks=5000, pt_range=(0.3, 50.0), pt_log=True, eta_max=2.5,
            noise_frac=0.2, chi2_cut=30.0, max_cands=6, max_holes=3, min_hits=4, dup_frac=0.5),
    3: dict(name="C3 batched build, barrel10, 256 events x log-uniform 200..8000 tracks",
            geom=geometry_barrel10, n_events=256, tracks=("loguniform", 200, 8000),
            pt_range=(0.5, 10.0), pt_log=False, eta_max=1.0, noise_frac=0.0, chi2_cut=30.0,
            max_cands=4, max_holes=3, min_hits=4, dup_frac=0.5),
    4: dict(name="C4 differentiated fit, barrel14, 100k tracks x 14 hits", geom=geometry_barrel14,
            n_events=1, tracks=100000, pt_range=(1.0, 10.0), pt_log=False, eta_max=0.8,
            noise_frac=0.0, chi2_cut=30.0, max_cands=4, max_holes=3, min_hits=4, dup_frac=0.5),
    5: dict(name="C5 stress, barrel10, 64 events x 10000 tracks, 50% noise", geom=geometry_barrel10,
            n_events=64, tracks=10000, pt_range=(0.3, 100.0), pt_log=True, eta_max=2.5,
            noise_frac=0.5, chi2_cut=30.0, max_cands=8, max_holes=3, min_hits=4, dup_frac=0.5),
}


def _n_tracks(spec, rng):
    t = spec["tracks"]
    if isinstance(t, tuple):
        _, lo, hi = t
        return int(np.exp(rng.uniform(np.log(lo), np.log(hi))))
    return int(t)


def make_config_event(config: int, event: int = 0, n_tracks=None, overlap_frac=0.0) -> Event:
    spec = WORKLOAD_SPECS[config]
    rng = np.random.default_rng(config_seed(config, event))
    n = _n_tracks(spec, rng) if n_tracks is None else int(n_tracks)
    return simulate_event(spec["geom"](), n, rng, pt_range=spec["pt_range"], pt_log=spec["pt_log"],
                          eta_max=spec["eta_max"], noise_frac=spec["noise_frac"], overlap_frac=overlap_frac)


def make_batch(config: int, n_events=None, n_tracks=None) -> EventBatch:
    spec = WORKLOAD_SPECS[config]
    E = spec["n_events"] if n_events is None else int(n_events)
    evs = [make_config_event(config, e, n_tracks) for e in range(E)]
    hoff = np.zeros(E + 1, np.int64)
    soff = np.zeros(E + 1, np.int64)
    hoff[1:] = np.cumsum([e.n_hits for e in evs])
    soff[1:] = np.cumsum([e.n_seeds for e in evs])
    return EventBatch(geom=evs[0].geom if evs else spec["geom"](), events=evs, hit_off=hoff,
                      seed_off=soff)
