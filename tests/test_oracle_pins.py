"""Pins of the FP64 oracle against facts that do not come from the oracle itself:
closed forms of helix motion, finite differences, linear-Gaussian identities,
brute-force enumeration, an independent truth simulation and pull statistics.

Each test names the property it relies on.  A plausible slip in the oracle
(a dropped term, a sign, a transposed Jacobian, a wrong index in the packed
covariance) fails at least one of them."""
import numpy as np
import pytest
from scipy.optimize import brentq, least_squares

import synth
from synth.events import ALPHA

BZ = 3.8


def geo_of(g):
    import oracle
    return oracle.Geo.of(g)


def rand_state(rng, kappa_range=(0.1, 1.5)):
    k = rng.uniform(*kappa_range) * rng.choice([-1, 1])
    return np.array([rng.normal(0, 0.3), rng.normal(0, 0.3), rng.normal(0, 2.0), k,
                     rng.uniform(-np.pi, np.pi), rng.uniform(0.6, 2.5)])


def rand_cov(rng, scale=(0.1, 0.1, 0.1, 0.02, 0.05, 0.05)):
    A = rng.normal(size=(6, 6)) * 0.3
    M = np.diag(np.square(scale)) + (A @ A.T) * np.outer(scale, scale) * 0.1
    import oracle
    return oracle.pack_cov(M)


# --- multiple scattering: the Highland width at hand-computed points --------

# theta0 = 0.0136 GeV / (beta p) sqrt(t) (1 + 0.038 ln t), pion mass 0.13957
# GeV, t = x/X0 / |cos(incidence)|; worked out by hand (to 12 digits) for:
#  A: p = 1 GeV, radial track through a barrel layer at normal incidence,
#     x/X0 = 0.01: beta = 0.990400134552, theta0 = 1.13288030327e-3;
#  B: p = 0.2 GeV, theta = pi/3 through a disk, x/X0 = 0.04, t = 0.08:
#     beta = 0.820059380940, theta0 = 2.12025333159e-2;
#  C: p = 3 GeV, theta = pi/4, radial in phi through a barrel layer,
#     x/X0 = 0.02, t = 0.02 / sin(pi/4) = 0.0282842712475:
#     beta = 0.998919543334, theta0 = 6.59828590496e-4.
# C_thetatheta grows by theta0^2 and C_phiphi by theta0^2 / sin^2(theta).
HIGHLAND_CASES = [
    # kind, pos, lo, hi, x0, (kappa, phi, theta), theta0^2, theta0^2 / sin^2 theta
    (0, 10.0, -50.0, 50.0, 0.01, (1.0, 0.0, np.pi / 2), 1.28341778153e-6, 1.28341778153e-6),
    (1, 20.0, 1.0, 100.0, 0.04, (5.77350269189626, 0.3, np.pi / 3), 4.49547419013e-4, 5.99396558684e-4),
    (0, 10.0, -50.0, 50.0, 0.02, (0.471404520791032, 0.0, np.pi / 4), 4.35373768836e-7, 8.70747537672e-7),
]


@pytest.mark.parametrize("case", range(len(HIGHLAND_CASES)))
def test_highland_width_at_hand_computed_points(orc, case):
    """With B = 0 the direction at the crossing is the start direction, so the
    material term the oracle adds at the layer is the Highland width of the
    hand-computed cases above, on C_thetatheta and (divided by sin^2 theta) on
    C_phiphi, and nothing else changes."""
    kind, pos, lo, hi, x0, (kappa, phi, theta), th2, phiphi = HIGHLAND_CASES[case]
    geo = orc.Geo(np.array([[kind, pos, lo, hi, x0]]), 0.0)
    p = np.array([0.0, 0.0, 0.0, kappa, phi, theta])
    C = orc.pack_cov(np.diag([1e-4, 1e-4, 1e-4, 1e-4, 1e-4, 1e-4]))
    _, c_mat, _ = orc.transport(geo, p, C, 0, +1, material=True)
    _, c_none, _ = orc.transport(geo, p, C, 0, +1, material=False)
    d = c_mat - c_none
    assert abs(d[orc.cov_index(5, 5)] - th2) <= 1e-10 * th2
    assert abs(d[orc.cov_index(4, 4)] - phiphi) <= 1e-10 * phiphi
    others = [k for k in range(21) if k not in (orc.cov_index(4, 4), orc.cov_index(5, 5))]
    assert np.all(d[others] == 0.0)


def test_joseph_update_keeps_realistic_fits_psd(orc):
    """The outward fits of the C2 event's true-hit tracks (pixel hits, strip
    disks with sigma_r / sigma_rphi = 333, fits that fail for loopers) end with
    covariances whose eigenvalues are >= -1e-12 of their trace: the Joseph-form
    update is a sum of positive semi-definite terms (the plain C - K R K^T left
    four of these indefinite)."""
    ev = synth.make_config_event(2)
    geo = geo_of(ev.geom)
    sel = (ev.true_hits >= 0).sum(1) >= 6
    _, cov, _, ok = orc.fit(geo, ev.hit_xyz, ev.hit_lcov, ev.hit_layer, ev.true_hits[sel], ev.seed_par[sel],
                            ev.seed_cov[sel])
    M = orc.unpack_cov(cov[ok == 1])
    w = np.linalg.eigvalsh(M)
    tr = np.trace(M, axis1=1, axis2=2)
    assert sel.sum() > 4000
    assert np.all(w[:, 0] >= -1e-12 * tr)


# --- helix closed forms ------------------------------------------------------

def test_helix_closure(orc):
    """After one full turn s = 2 pi/|omega| the transverse position returns and
    z advances by 2 pi cot(theta)/|omega|."""
    rng = np.random.default_rng(1)
    for _ in range(20):
        p = rand_state(rng)
        om = -ALPHA * BZ * p[3]
        s = 2 * np.pi / abs(om)
        q = orc.helix(BZ, p, s)
        R = 1 / abs(om)
        assert abs(q[0] - p[0]) < 1e-12 * R and abs(q[1] - p[1]) < 1e-12 * R
        assert abs(q[2] - (p[2] + s * np.cos(p[5]) / np.sin(p[5]))) < 1e-10 * (1 + abs(q[2]))
        assert abs(abs(q[4] - p[4]) - 2 * np.pi) < 1e-12


def test_helix_straight_line_limit(orc):
    """B = 0 is the straight line exactly; for a weak field the deviation from
    the line is (omega s^2 / 2) along the left normal to first order."""
    rng = np.random.default_rng(2)
    for _ in range(20):
        p = rand_state(rng)
        s = rng.uniform(1, 100)
        q = orc.helix(0.0, p, s)
        line = p[:3] + s * np.array([np.cos(p[4]), np.sin(p[4]), np.cos(p[5]) / np.sin(p[5])])
        assert np.allclose(q[:3], line, rtol=0, atol=1e-12 * (1 + np.abs(line).max()))
        bz = 1e-6
        q = orc.helix(bz, p, s)
        om = -ALPHA * bz * p[3]
        exp = 0.5 * om * s * s * np.array([-np.sin(p[4]), np.cos(p[4])])
        dev = q[:2] - line[:2]
        assert np.linalg.norm(dev - exp) < 1e-4 * np.linalg.norm(exp)


def _xy_at(p, s, bz):
    """Independent helix form (not the sinc form): circle through the start."""
    om = -ALPHA * bz * p[3]
    return (p[0] + (np.sin(p[4] + om * s) - np.sin(p[4])) / om,
            p[1] - (np.cos(p[4] + om * s) - np.cos(p[4])) / om)


def test_cylinder_path_is_first_crossing(orc):
    """The returned s solves r(s) = r_L to 1e-12 relative and no smaller s > 0
    reaches the cylinder (scan from inside)."""
    g = synth.geometry_barrel10()
    geo = geo_of(g)
    rng = np.random.default_rng(3)
    n = 0
    for _ in range(60):
        p = rand_state(rng)
        p[:3] = 0.0
        for l in range(g.n_layers):
            s, q = orc.path(geo, p, l, +1)
            if s is None:
                # unreachable: the particle's circle (diameter 2/|omega| through the origin) is too small
                om = -ALPHA * BZ * p[3]
                assert 2 / abs(om) < g.pos[l] * (1 + 1e-9)
                continue
            n += 1
            x, y = _xy_at(p, s, BZ)
            assert abs(np.hypot(x, y) - g.pos[l]) < 1e-12 * g.pos[l]
            grid = np.linspace(0, s, 2001)[1:-1]
            xs, ys = _xy_at(p, grid, BZ)
            assert np.all(np.hypot(xs, ys) < g.pos[l])
    assert n > 200


def test_plane_path(orc):
    g = synth.geometry_cmslike()
    geo = geo_of(g)
    rng = np.random.default_rng(4)
    for _ in range(50):
        p = rand_state(rng)
        l = int(rng.integers(14, g.n_layers))
        s, q = orc.path(geo, p, l, +1)
        zl = g.pos[l]
        cot = np.cos(p[5]) / np.sin(p[5])
        if (zl - p[2]) * cot > 0:
            assert s is not None and s > 0
            assert abs(q[2] - zl) < 1e-12 * abs(zl)
        else:
            assert s is None


# --- Jacobian ----------------------------------------------------------------

def _prop_fd(orc, geo, p, layer, direction=+1):
    s, q = orc.path(geo, p, layer, direction)
    return q


@pytest.mark.parametrize("geom_name,layer", [("barrel10", 3), ("barrel10", 8), ("cmslike", 20), ("cmslike", 30)])
def test_jacobian_vs_central_differences(orc, geom_name, layer):
    """J (forward-mode derivative incl. ds/dp) equals FP64 central differences
    of the oracle's own propagator p -> helix(p, s*(p))."""
    g = synth.geometry_barrel10() if geom_name == "barrel10" else synth.geometry_cmslike()
    geo = geo_of(g)
    rng = np.random.default_rng(5 + layer)
    C = rand_cov(rng)
    done = 0
    for _ in range(40):
        p = rand_state(rng, (0.1, 0.8))
        if g.kind[layer] == 1:
            p[5] = rng.uniform(0.2, 0.5) if g.pos[layer] > 0 else rng.uniform(2.6, 2.9)
        res = orc.transport(geo, p, C, layer)
        if res is None:
            continue
        _, _, J = res
        Jfd = np.zeros((6, 6))
        for j in range(6):
            h = 1e-6 * max(1.0, abs(p[j]))
            pp, pm = p.copy(), p.copy()
            pp[j] += h
            pm[j] -= h
            qp = _prop_fd(orc, geo, pp, layer)
            qm = _prop_fd(orc, geo, pm, layer)
            d = qp - qm
            d[4] = (d[4] + np.pi) % (2 * np.pi) - np.pi
            Jfd[:, j] = d / (2 * h)
        scale = np.maximum(1.0, np.abs(J))
        assert np.max(np.abs(J - Jfd) / scale) < 1e-6, (J, Jfd)
        done += 1
    assert done >= 10


def test_surface_null_vector_and_psd(orc):
    """After transport onto a cylinder the position component normal to it has
    zero variance (C n = 0, n = (x, y, 0, ...)/r); onto a plane, C e_z = 0; C
    stays symmetric positive semi-definite (rank 5)."""
    import oracle
    rng = np.random.default_rng(6)
    for geom, layers in ((synth.geometry_barrel10(), range(10)), (synth.geometry_cmslike(), range(14, 38))):
        geo = geo_of(geom)
        for _ in range(30):
            p = rand_state(rng, (0.05, 0.6))
            l = int(rng.choice(list(layers)))
            C = rand_cov(rng)
            res = orc.transport(geo, p, C, l, material=True)
            if res is None:
                continue
            q, C2, _ = res
            M = oracle.unpack_cov(C2)
            if geom.kind[l] == 0:
                n = np.array([q[0], q[1], 0, 0, 0, 0]) / np.hypot(q[0], q[1])
            else:
                n = np.array([0, 0, 1.0, 0, 0, 0])
            assert np.linalg.norm(M @ n) < 1e-10 * np.linalg.norm(M)
            ev = np.linalg.eigvalsh(M)
            assert ev.min() > -1e-12 * np.trace(M)


def test_round_trip_and_inverse_jacobian(orc):
    """A -> B -> A restores the state; J_BA J_AB is the identity on the tangent
    space of surface A."""
    import oracle
    g = synth.geometry_barrel10()
    geo = geo_of(g)
    rng = np.random.default_rng(7)
    C = rand_cov(rng)
    n = 0
    for _ in range(30):
        p0 = rand_state(rng, (0.05, 0.5))
        p0[:3] = 0
        a = orc.transport(geo, p0, C, 2)
        if a is None:
            continue
        pa, Ca, _ = a
        b = orc.transport(geo, pa, Ca, 7, +1)
        if b is None:
            continue
        pb, Cb, Jab = b
        c = orc.transport(geo, pb, Cb, 2, -1)
        assert c is not None
        pa2, Ca2, Jba = c
        d = pa2 - pa
        d[4] = (d[4] + np.pi) % (2 * np.pi) - np.pi
        assert np.max(np.abs(d)) < 1e-10 * (1 + np.abs(pa).max())
        assert np.allclose(oracle.unpack_cov(Ca2), oracle.unpack_cov(Ca), rtol=1e-8, atol=1e-12)
        nA = np.array([pa[0], pa[1], 0, 0, 0, 0]) / np.hypot(pa[0], pa[1])
        for _ in range(4):
            v = rng.normal(size=6)
            v -= nA * (nA @ v)
            w = Jba @ (Jab @ v)
            assert np.linalg.norm(w - v) < 1e-8 * np.linalg.norm(v)
        n += 1
    assert n >= 10


# --- Kalman update -----------------------------------------------------------

def _H_from_geometry(kind, hit):
    """Measurement rows from the surface geometry at the hit: the unit tangent
    of the circle through the hit, and the axis (barrel) or the outward radial
    direction (disk)."""
    phi = np.arctan2(hit[1], hit[0])
    t = np.array([-np.sin(phi), np.cos(phi), 0, 0, 0, 0])
    b = np.array([0, 0, 1.0, 0, 0, 0]) if kind == 0 else np.array([np.cos(phi), np.sin(phi), 0, 0, 0, 0])
    m = np.array([0.0, hit[2] if kind == 0 else np.hypot(hit[0], hit[1])])
    return np.stack([t, b]), m


@pytest.mark.parametrize("kind", [0, 1])
def test_update_information_form(orc, kind):
    """From a positive-definite prior, the update equals Gaussian conditioning
    in information form: C'^-1 = C^-1 + H^T V^-1 H, C'^-1 p' = C^-1 p + H^T V^-1 m;
    chi2 = min over q of |q - p|^2_C + |m - H q|^2_V; C' symmetric PSD."""
    import oracle
    rng = np.random.default_rng(10 + kind)
    for _ in range(20):
        p = rand_state(rng)
        C = rand_cov(rng)
        M = oracle.unpack_cov(C)
        phi = p[4] + rng.normal(0, 0.02)
        r = 30.0
        hit = np.array([r * np.cos(phi), r * np.sin(phi), p[2] + rng.normal(0, 0.1)])
        p[0], p[1] = (r + rng.normal(0, 0.05)) * np.cos(phi + 0.003), (r + rng.normal(0, 0.05)) * np.sin(phi + 0.003)
        lc = np.array([0.01 ** 2, 0.02 ** 2, 0.3 * 0.01 * 0.02])
        chi2, p2, C2 = orc.update(kind, p, C, hit, lc)
        H, m = _H_from_geometry(kind, hit)
        V = np.array([[lc[0], lc[2]], [lc[2], lc[1]]])
        Ci = np.linalg.inv(M)
        Vi = np.linalg.inv(V)
        info = Ci + H.T @ Vi @ H
        M2 = oracle.unpack_cov(C2)
        assert np.allclose(np.linalg.inv(info), M2, rtol=1e-7, atol=1e-12 * np.abs(M).max())
        mean = np.linalg.solve(info, Ci @ p + H.T @ Vi @ m)
        d = p2 - mean
        d[4] = (d[4] + np.pi) % (2 * np.pi) - np.pi
        assert np.max(np.abs(d)) < 1e-9 * (1 + np.abs(p).max())
        obj = (mean - p) @ Ci @ (mean - p) + (m - H @ mean) @ Vi @ (m - H @ mean)
        assert abs(chi2 - obj) < 1e-8 * (1 + obj)
        assert np.linalg.eigvalsh(M2).min() > -1e-14


def test_update_zero_residual(orc):
    """A state sitting on the hit with the hit's direction gives chi2 = 0 and an
    unchanged parameter vector."""
    rng = np.random.default_rng(12)
    for kind in (0, 1):
        p = rand_state(rng)
        r = 20.0
        p[0], p[1] = r * np.cos(0.7), r * np.sin(0.7)
        hit = np.array([p[0], p[1], p[2]])
        chi2, p2, _ = orc.update(kind, p, rand_cov(rng), hit, np.array([1e-4, 1e-4, 0]))
        assert chi2 < 1e-20
        assert np.allclose(p2, p, rtol=0, atol=1e-12)


# --- fit vs brute-force weighted least squares ---------------------------------

def _line_plane(p, z):
    t = (z - p[2]) * np.tan(p[5])
    return np.array([p[0] + t * np.cos(p[4]), p[1] + t * np.sin(p[4]), z])


def _helix_cyl(p, r, bz):
    om = -ALPHA * bz * p[3]

    def f(s):
        x, y = _xy_at(p, s, bz)
        return x * x + y * y - r * r

    s = brentq(f, 0.0, (np.pi * 0.999) / abs(om), xtol=1e-15, rtol=1e-15)
    x, y = _xy_at(p, s, bz)
    return np.array([x, y, p[2] + s * np.cos(p[5]) / np.sin(p[5])])


def _local_residual(kind, pt, hit):
    phi = np.arctan2(hit[1], hit[0])
    ra = np.sin(phi) * pt[0] - np.cos(phi) * pt[1]
    rb = (hit[2] - pt[2]) if kind == 0 else (np.hypot(hit[0], hit[1]) - (np.cos(phi) * pt[0] + np.sin(phi) * pt[1]))
    return np.array([ra, rb])


@pytest.mark.parametrize("case", ["planes_B0", "cylinders_B38"])
def test_fit_equals_weighted_least_squares(orc, case):
    """Without material the forward Kalman fit is the maximum-a-posteriori
    estimate of the start state given the seed prior and all hits (linear
    Gaussian identity, here to linearisation accuracy with a tight prior):
    its final state equals the least-squares optimum transported to the last
    surface, and the sum of predicted chi2 equals the optimum's objective."""
    import oracle
    rng = np.random.default_rng(20)
    if case == "planes_B0":
        bz = 0.0
        zs = np.linspace(10, 100, 8)
        g = synth.Geometry(kind=np.ones(8, np.int32), pos=zs, lo=np.zeros(8), hi=np.full(8, 200.0),
                           x0=np.zeros(8), sig_a=np.full(8, 0.01), sig_b=np.full(8, 0.02), bz=0.0)
    else:
        bz = 3.8
        rs = np.linspace(4, 60, 8)
        g = synth.Geometry(kind=np.zeros(8, np.int32), pos=rs, lo=np.full(8, -300.0), hi=np.full(8, 300.0),
                           x0=np.zeros(8), sig_a=np.full(8, 0.01), sig_b=np.full(8, 0.02), bz=bz)
    geo = oracle.Geo(g.table(), bz)
    sig_prior = np.array([1e-4, 1e-4, 1e-4, 1e-4, 2e-5, 2e-5])   # tight: linearisation error ~ sigma^2
    for trial in range(5):
        true = np.array([0, 0, 0, rng.choice([-1, 1]) * rng.uniform(0.2, 1.0), rng.uniform(-3, 3),
                         rng.uniform(0.3, 0.6) if case == "planes_B0" else rng.uniform(1.0, 2.0)])
        seed = true + rng.normal(size=6) * sig_prior
        P = np.diag(sig_prior ** 2)
        if case == "planes_B0":
            pts = [_line_plane(true, z) for z in g.pos]
        else:
            pts = [_helix_cyl(true, r, bz) for r in g.pos]
        hits, lcov = [], []
        for k, pt in enumerate(pts):
            phi = np.arctan2(pt[1], pt[0])
            if case == "planes_B0":
                rr = np.hypot(pt[0], pt[1]) + rng.normal(0, 0.02)
                ph = phi + rng.normal(0, 0.01) / np.hypot(pt[0], pt[1])
                hits.append([rr * np.cos(ph), rr * np.sin(ph), pt[2]])
            else:
                ph = phi + rng.normal(0, 0.01) / g.pos[k]
                hits.append([g.pos[k] * np.cos(ph), g.pos[k] * np.sin(ph), pt[2] + rng.normal(0, 0.02)])
            lcov.append([0.01 ** 2, 0.02 ** 2, 0.0])
        hits = np.array(hits); lcov = np.array(lcov)
        hl = np.arange(8, dtype=np.int32)
        par, cov, chi2, ok = orc.fit(geo, hits, lcov, hl, hl[None, :], seed[None], oracle.pack_cov(P)[None])
        assert ok[0] == 1
        Lp = np.linalg.cholesky(np.linalg.inv(P))

        def resid(q):
            out = [Lp.T @ (q - seed)]
            for k in range(8):
                pt = _line_plane(q, g.pos[k]) if case == "planes_B0" else _helix_cyl(q, g.pos[k], bz)
                out.append(_local_residual(g.kind[k], pt, hits[k]) / np.array([0.01, 0.02]))
            return np.concatenate(out)

        sol = least_squares(resid, seed, xtol=1e-15, ftol=1e-15, gtol=1e-15, x_scale=sig_prior)
        obj = float(np.sum(sol.fun ** 2))
        last = oracle.transport(geo, sol.x, oracle.pack_cov(P), 7)[0]
        sig = np.sqrt(np.diag(oracle.unpack_cov(cov[0])))
        d = par[0] - last
        d[4] = (d[4] + np.pi) % (2 * np.pi) - np.pi
        on = sig > 1e-9
        assert np.max(np.abs(d[on]) / sig[on]) < 1e-3, (d, sig)
        assert abs(chi2[0] - obj) < 1e-3 * max(1.0, obj)


# --- combinatorial search vs exhaustive enumeration -----------------------------

def _tiny_event(rng, n_layers=4, fakes=2):
    g = synth.Geometry(kind=np.zeros(n_layers, np.int32), pos=np.linspace(5, 30, n_layers),
                       lo=np.full(n_layers, -100.0), hi=np.full(n_layers, 100.0), x0=np.full(n_layers, 0.01),
                       sig_a=np.full(n_layers, 0.01), sig_b=np.full(n_layers, 0.01), bz=3.8)
    ev = synth.simulate_event(g, 1, rng, pt_range=(1.0, 3.0), eta_max=0.5)
    xyz = [ev.hit_xyz]
    lay = [ev.hit_layer]
    for h in range(ev.n_hits):
        for _ in range(fakes):
            r = g.pos[ev.hit_layer[h]]
            ph = np.arctan2(ev.hit_xyz[h, 1], ev.hit_xyz[h, 0]) + rng.normal(0, 0.03 / r * 3)
            xyz.append(np.array([[r * np.cos(ph), r * np.sin(ph), ev.hit_xyz[h, 2] + rng.normal(0, 0.03)]]))
            lay.append(np.array([ev.hit_layer[h]], np.int32))
    xyz = np.concatenate(xyz); lay = np.concatenate(lay)
    lc = np.tile([1e-4, 1e-4, 0.0], (xyz.shape[0], 1))
    seed_cov = ev.seed_cov.copy()
    return g, xyz, lc, lay, ev.seed_par, seed_cov


def _enumerate(orc, geo, g, xyz, lc, lay, p, C, cut, max_holes):
    """All leaves of the search tree with (score, hits); a leaf is a candidate
    with no next surface or no admissible child."""
    leaves = []

    def rec(p, C, score, nholes, rho, hits):
        l, s = orc.next_surface(geo, p, rho, 0.0)
        if l < 0:
            leaves.append((score, tuple(hits)))
            return
        pr, Cr, _ = orc.transport(geo, p, C, l, material=True)
        kids = 0
        for h in np.nonzero(lay == l)[0]:
            chi2, p2, C2 = orc.update(0, pr, Cr, xyz[h], lc[h])
            phi = np.arctan2(xyz[h, 1], xyz[h, 0])
            if np.cos(phi) * pr[0] + np.sin(phi) * pr[1] <= 0:
                continue
            if chi2 < cut:
                kids += 1
                rec(p2, C2, score + 10 - chi2, nholes, g.pos[l], hits + [int(h)])
        if nholes + 1 <= max_holes:
            kids += 1
            rec(pr, Cr, score - 10, nholes + 1, g.pos[l], hits + [-1])
        if kids == 0:
            leaves.append((score, tuple(hits)))

    rec(p, C, 0.0, 0, 0.0, [])
    return leaves


def test_search_equals_exhaustive_enumeration(orc):
    """With a per-seed cap larger than the search tree, the kept track is the
    best-scoring leaf of the exhaustive tree; with a cap of 1 it is the greedy
    path."""
    import oracle
    rng = np.random.default_rng(30)
    for trial in range(6):
        g, xyz, lc, lay, sp, sc = _tiny_event(rng)
        geo = oracle.Geo.of(g)
        leaves = _enumerate(orc, geo, g, xyz, lc, lay, sp[0], sc[0], 30.0, 1)
        best = max(leaves, key=lambda t: t[0])
        out = orc.build_event(geo, xyz, lc, lay, sp, sc, chi2_cut=30.0, max_cands=512, max_holes=1, min_hits=1)
        n = out["nsteps"][0]
        assert tuple(out["hits"][0][:n].tolist()) == best[1]
        assert abs(out["score"][0] - best[0]) < 1e-9
        # greedy
        p, C, rho, hits, score, nholes = sp[0], sc[0], 0.0, [], 0.0, 0
        while True:
            l, _ = orc.next_surface(geo, p, rho, 0.0)
            if l < 0:
                break
            pr, Cr, _ = orc.transport(geo, p, C, l, material=True)
            opts = []
            for h in np.nonzero(lay == l)[0]:
                chi2, p2, C2 = orc.update(0, pr, Cr, xyz[h], lc[h])
                if chi2 < 30.0:
                    opts.append((score + 10 - chi2, int(h), p2, C2))
            if nholes + 1 <= 1:
                opts.append((score - 10, 1 << 30, pr, Cr))
            if not opts:
                break
            sc_, h, p, C = max(opts, key=lambda o: (o[0], -o[1]))
            score = sc_
            if h == 1 << 30:
                nholes += 1
                hits.append(-1)
            else:
                hits.append(h)
            rho = g.pos[l]
        out1 = orc.build_event(geo, xyz, lc, lay, sp, sc, chi2_cut=30.0, max_cands=1, max_holes=1, min_hits=1)
        n1 = out1["nsteps"][0]
        assert out1["hits"][0][:n1].tolist() == hits
        assert abs(out1["score"][0] - score) < 1e-9


def test_navigation_matches_independent_truth_simulation(orc):
    """Stepping the true (unscattered) helix with the oracle's navigation visits
    the same surfaces as the independent truth simulation, CMS-like geometry."""
    import oracle
    g = synth.geometry_cmslike()
    geo = oracle.Geo.of(g)
    rng = np.random.default_rng(40)
    ev = synth.simulate_event(g, 300, rng, pt_range=(0.3, 50), pt_log=True, eta_max=2.5, kick=False)
    agree = 0
    C = np.zeros(21)
    for t in range(ev.n_seeds):
        p = ev.true_par[t].copy()
        rho, zeta, seq = 0.0, 0.0, []
        while True:
            l, s = orc.next_surface(geo, p, rho, zeta)
            if l < 0:
                break
            p, _, _ = orc.transport(geo, p, C, l)
            seq.append(l)
            if g.kind[l] == 0:
                rho, zeta = g.pos[l], max(zeta, abs(p[2]))
            else:
                zeta, rho = abs(g.pos[l]), max(rho, np.hypot(p[0], p[1]))
        truth = ev.true_layers[t][ev.true_layers[t] >= 0].tolist()
        agree += seq == truth
    assert agree >= 0.99 * ev.n_seeds


def test_efficiency_config1(orc):
    """Sec. 3 matching (more than 75 % of a track's hits from one simulated
    particle): building efficiency close to 1 on the noiseless barrel event."""
    import oracle
    ev = synth.make_config_event(1)
    geo = oracle.Geo.of(ev.geom)
    out = orc.build_event(geo, ev.hit_xyz, ev.hit_lcov, ev.hit_layer, ev.seed_par, ev.seed_cov, max_cands=4)
    eff = 0
    for s in range(ev.n_seeds):
        hs = out["hits"][s][out["hits"][s] >= 0]
        if len(hs) and (ev.hit_track[hs] == s).sum() > 0.75 * len(hs):
            eff += 1
    assert eff >= 0.95 * ev.n_seeds


# --- duplicate removal ------------------------------------------------------

def test_dedup_hand_built(orc):
    L = 6
    def row(*h):
        return list(h) + [-1] * (L - len(h))
    hits = np.array([row(1, 2, 3, 4),        # 0: score 50
                     row(1, 2, 3, 9),        # 1: 40, shares 3/4 with 0 -> duplicate
                     row(1, 2, 10, 11),      # 2: 45, shares 2/4 with 0 -> kept (not > 0.5)
                     row(10, 11, 12, 13),    # 3: 30, shares 2/4 with 2 -> kept
                     row(20, 21, 22),        # 4: 60 but only 3 hits -> short
                     row(30, 31, 32, 33, 34),  # 5: 20
                     row(30, 31, 32, 33, 34),  # 6: 20, identical to 5, higher seed id -> duplicate
                     row(10, 11, 12, 40)])   # 7: 35, shares 3/4 with 3 only after 3 kept? 3 has 30 < 35
    score = np.array([50, 40, 45, 30, 60, 20, 20, 35.0])
    nh = np.array([4, 4, 4, 4, 3, 5, 5, 4])
    flags = orc.dedup(hits, score, nh, min_hits=4, dup_frac=0.5)
    # order: 0(50) 2(45) 1(40) 7(35) 3(30) 5(20) 6(20)
    # 7 shares {10,11} with 2 (2/4, kept); 3 shares {10,11,12} with 7 (3/4) -> duplicate
    assert flags.tolist() == [1, 2, 1, 2, 0, 1, 2, 1]


# --- statistics: pulls and chi2 --------------------------------------------------

@pytest.mark.slow
def test_fit_pulls_and_chi2(orc):
    """Consistency of the model with the simulation: fitted minus true state at
    the last crossing, divided by the fitted sigma, is N(0,1) in each local
    coordinate, and sum chi2 / (2 n_hits) is 1 (10^4 tracks, 14 barrel layers)."""
    import oracle
    g = synth.geometry_barrel14()
    geo = oracle.Geo.of(g)
    rng = np.random.default_rng(50)
    ev = synth.simulate_event(g, 10000, rng, pt_range=(1.0, 10.0), eta_max=0.8)
    nt = (ev.true_hits >= 0).sum(1)
    sel = np.nonzero(nt == 14)[0]
    # the seed's position prior (0.1 cm) is honoured by smearing it too, so that
    # every term of the prior is statistically consistent
    sp = ev.seed_par[sel].copy()
    sp[:, :3] += rng.normal(0, 0.1, (len(sel), 3))
    par, cov, chi2, ok = orc.fit(geo, ev.hit_xyz, ev.hit_lcov, ev.hit_layer, ev.true_hits[sel],
                                 sp, ev.seed_cov[sel])
    assert ok.all()
    tru = ev.true_state[sel, 13]
    M = oracle.unpack_cov(cov)
    phic = np.arctan2(tru[:, 1], tru[:, 0])
    t = np.stack([-np.sin(phic), np.cos(phic)], 1)
    d_rphi = np.einsum("ij,ij->i", par[:, :2] - tru[:, :2], t)
    v_rphi = np.einsum("ni,nij,nj->n", t, M[:, :2, :2], t)
    pulls = {"rphi": d_rphi / np.sqrt(v_rphi)}
    for name, k in (("z", 2), ("kappa", 3), ("phi", 4), ("theta", 5)):
        d = par[:, k] - tru[:, k]
        if k == 4:
            d = (d + np.pi) % (2 * np.pi) - np.pi
        pulls[name] = d / np.sqrt(M[:, k, k])
    for name, pl in pulls.items():
        assert abs(pl.mean()) < 0.05, (name, pl.mean())
        assert abs(pl.std() - 1) < 0.06, (name, pl.std())
    r = chi2.sum() / (2 * 14 * len(sel))
    assert abs(r - 1) < 0.03, r


# --- reference gradient ------------------------------------------------------------

def test_gradient_vs_central_differences(orc):
    """Dual-number gradient of the fit objective against FP64 central
    differences (h = 1e-6) for hit positions, alignment and thickness."""
    import oracle
    g = synth.geometry_barrel14()
    geo = oracle.Geo.of(g)
    rng = np.random.default_rng(60)
    ev = synth.simulate_event(g, 4, rng, pt_range=(1.0, 5.0), eta_max=0.8)
    hits = ev.true_hits
    keep = (hits >= 0).sum(1) == 14
    hits, sp, sc = hits[keep], ev.seed_par[keep], ev.seed_cov[keep]
    T = hits.shape[0]
    gchi = rng.normal(size=T)
    gpar = rng.normal(size=(T, 6))
    align = rng.normal(0, 1e-3, (g.n_layers, 3))
    x0 = g.x0 * (1 + 0.1 * rng.random(g.n_layers))
    gh, ga, gx = orc.fit_grad(geo, ev.hit_xyz, ev.hit_lcov, ev.hit_layer, hits, sp, sc, gchi, g_par=gpar,
                              align=align, x0=x0)

    def loss(hx=None, al=None, xx=None):
        par, cov, chi2, ok = orc.fit(geo, ev.hit_xyz if hx is None else hx, ev.hit_lcov, ev.hit_layer, hits, sp, sc,
                                     align=align if al is None else al, x0=x0 if xx is None else xx)
        return float(gchi @ chi2 + np.sum(gpar * par))

    def fd(kind, idx):
        h = 1e-6
        if kind == "hit":
            a = ev.hit_xyz.copy(); b = a.copy()
            a[idx] += h * max(1, abs(a[idx])); b[idx] -= h * max(1, abs(b[idx]))
            return (loss(hx=a) - loss(hx=b)) / (2 * h * max(1, abs(ev.hit_xyz[idx])))
        if kind == "align":
            a = align.copy(); b = a.copy(); a[idx] += h; b[idx] -= h
            return (loss(al=a) - loss(al=b)) / (2 * h)
        # x/X0 ~ 0.01 enters the loss only through the scattering variance: a
        # 1e-6 step moves the loss by ~1e-11 of itself, the size of its FP64
        # rounding, so the step is 1e-4 (1 % of x/X0) with the five-point
        # stencil, whose truncation is O(h^4)
        hx = 1e-4

        def at(k):
            a = x0.copy()
            a[idx] += k * hx
            return loss(xx=a)
        return (-at(2) + 8 * at(1) - 8 * at(-1) + at(-2)) / (12 * hx)

    used = np.unique(hits[hits >= 0])
    checks = [("hit", (int(h), c)) for h in rng.choice(used, 6, replace=False) for c in range(3)]
    checks += [("align", (l, c)) for l in (0, 5, 13) for c in range(3)]
    checks += [("x0", l) for l in (0, 7, 13)]
    for kind, idx in checks:
        ref = fd(kind, idx)
        got = gh[idx] if kind == "hit" else (ga[idx] if kind == "align" else gx[idx])
        assert abs(got - ref) <= 1e-6 * max(1.0, abs(ref)), (kind, idx, got, ref)


@pytest.mark.slow
def test_backward_fit_pulls(orc):
    """The inward fit (from the outward result, covariance reset to 100 x the
    seed diagonal) estimates the state at the innermost hit: position at the
    first crossing and the direction before the first scattering (the vertex
    direction) with N(0,1) pulls."""
    import oracle
    g = synth.geometry_barrel14()
    geo = oracle.Geo.of(g)
    rng = np.random.default_rng(51)
    ev = synth.simulate_event(g, 6000, rng, pt_range=(1.0, 10.0), eta_max=0.8)
    sel = np.nonzero((ev.true_hits >= 0).sum(1) == 14)[0]
    hits = ev.true_hits[sel]
    par, cov, chi2, ok = orc.fit(geo, ev.hit_xyz, ev.hit_lcov, ev.hit_layer, hits, ev.seed_par[sel], ev.seed_cov[sel])
    bpar, bcov, bchi2, bok = orc.fit(geo, ev.hit_xyz, ev.hit_lcov, ev.hit_layer, hits, par, cov, direction=-1)
    assert bok.all()
    M = oracle.unpack_cov(bcov)
    tru = np.concatenate([ev.true_state[sel, 0, :3], ev.true_par[sel, 3:]], 1)
    # direction just before the first layer: the vertex azimuth turned by omega*s0
    # along the arc of chord |P0| (circle through the origin)
    om = -ALPHA * g.bz * tru[:, 3]
    chord = np.hypot(tru[:, 0], tru[:, 1])
    s0 = 2.0 / np.abs(om) * np.arcsin(chord * np.abs(om) / 2)
    tru[:, 4] = tru[:, 4] + om * s0
    phic = np.arctan2(tru[:, 1], tru[:, 0])
    t = np.stack([-np.sin(phic), np.cos(phic)], 1)
    pulls = {"rphi": np.einsum("ij,ij->i", bpar[:, :2] - tru[:, :2], t)
             / np.sqrt(np.einsum("ni,nij,nj->n", t, M[:, :2, :2], t))}
    for name, k in (("z", 2), ("kappa", 3), ("phi", 4), ("theta", 5)):
        d = bpar[:, k] - tru[:, k]
        if k == 4:
            d = (d + np.pi) % (2 * np.pi) - np.pi
        pulls[name] = d / np.sqrt(M[:, k, k])
    for name, pl in pulls.items():
        assert abs(pl.mean()) < 0.06, (name, pl.mean())
        assert abs(pl.std() - 1) < 0.08, (name, pl.std())


def test_fit_skips_empty_slots_and_keeps_empty_rows(orc):
    """Fitting applies the KF to the hits found (Sec. 1), so an empty slot (-1)
    is no step: a row with empty slots between its hits fits exactly like the
    same hits packed together, in both directions.  A row with no hit leaves
    the start untouched: forward, the given state and covariance; inward, the
    given state with the reset prior (100 x the seed-style diagonal
    0.01, 0.01, 0.01 cm^2, (0.05 kappa)^2, 0.0025, 0.0025), chi2 0."""
    import oracle
    g = synth.geometry_barrel14()
    geo = oracle.Geo.of(g)
    rng = np.random.default_rng(61)
    ev = synth.simulate_event(g, 200, rng, pt_range=(1.0, 10.0), eta_max=0.8)
    sel = np.nonzero((ev.true_hits >= 0).sum(1) == 14)[0][:40]
    packed = ev.true_hits[sel].copy()
    sp, sc = ev.seed_par[sel], ev.seed_cov[sel]
    T, K = packed.shape
    keep = rng.random((T, K)) < 0.6
    keep[:, 0] = True
    gappy = np.full((T, 2 * K), -1, np.int32)
    compact = np.full((T, K), -1, np.int32)
    for t in range(T):
        h = packed[t][keep[t]]
        compact[t, :len(h)] = h
        slots = np.sort(rng.choice(2 * K, len(h), replace=False))
        gappy[t, slots] = h
    fa = orc.fit(geo, ev.hit_xyz, ev.hit_lcov, ev.hit_layer, gappy, sp, sc)
    fb = orc.fit(geo, ev.hit_xyz, ev.hit_lcov, ev.hit_layer, compact, sp, sc)
    for x, y in zip(fa, fb):
        assert np.array_equal(x, y)
    ba = orc.fit(geo, ev.hit_xyz, ev.hit_lcov, ev.hit_layer, gappy, fa[0], fa[1], direction=-1)
    bb = orc.fit(geo, ev.hit_xyz, ev.hit_lcov, ev.hit_layer, compact, fa[0], fa[1], direction=-1)
    for x, y in zip(ba, bb):
        assert np.array_equal(x, y)
    empty = np.full((T, K), -1, np.int32)
    par, cov, chi2, ok = orc.fit(geo, ev.hit_xyz, ev.hit_lcov, ev.hit_layer, empty, sp, sc)
    assert np.array_equal(par, sp) and np.array_equal(cov, sc) and (chi2 == 0).all() and ok.all()
    par, cov, chi2, ok = orc.fit(geo, ev.hit_xyz, ev.hit_lcov, ev.hit_layer, empty, sp, sc, direction=-1)
    assert np.array_equal(par, sp) and (chi2 == 0).all() and ok.all()
    prior = np.zeros((T, 6, 6))
    for i, d in enumerate((0.01, 0.01, 0.01, 0.0, 0.0025, 0.0025)):
        prior[:, i, i] = 100.0 * d
    prior[:, 3, 3] = 100.0 * (0.05 * sp[:, 3]) ** 2
    assert np.allclose(oracle.unpack_cov(cov), prior, rtol=1e-15, atol=0)
