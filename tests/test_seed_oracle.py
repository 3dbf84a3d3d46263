"""Pins of the hit-based seeding oracle (Sec. 3: seeds from the four innermost
barrel layers, prompt tracks) against facts that do not come from it:
  * hits placed exactly on helices from the beam line (the simulation's own
    helix and cylinder-crossing code, not the oracle's) give exactly their
    quadruplet, with the helix's z0, kappa, phi and theta;
  * the cut margins follow closed forms: 1 - pt_min / pT for the curvature,
    1 - |z0| / z_max, 1 - R3 |sin d| / rphi_tol for a hit turned by d about
    the axis on the last layer, 1 - |dz| / z_tol for one moved in z;
  * rotating the event about z, mirroring it in z or in y maps the seeds as
    the symmetry says (same quadruplets; phi + a; z0, theta -> -z0, pi -
    theta; kappa, phi -> -kappa, -phi)."""
import numpy as np
import pytest

import oracle
import synth.events as sev
from synth.geometry import geometry_cmslike

ALPHA = 0.00299792458
CUTS = dict(pt_min=0.5, z_max=5.0, rphi_tol=0.05, z_tol=0.1)


def _track_hits(geo, z0, kappa, phi, theta):
    """The four seeding-layer crossings of an exact helix from (0, 0, z0)."""
    ids, radii = oracle.seeding_layers(geo)
    omega = -ALPHA * geo.bz * kappa
    cot = 1.0 / np.tan(theta)
    out = []
    for r in radii:
        s = sev._cylinder_path(np.array([0.0]), np.array([0.0]), np.array([phi]), np.array([omega]), r)[0]
        x, y, z = sev._position_at(0.0, 0.0, z0, phi, cot, omega, s)
        out.append((x, y, z))
    return np.array(out), ids


def _event(geo, tracks):
    xyz, lay = [], []
    for t in tracks:
        p, ids = _track_hits(geo, *t)
        xyz.append(p)
        lay.append(ids)
    return np.concatenate(xyz), np.concatenate(lay).astype(np.int32)


TRACKS = [(0.3, 1.0 / 0.8, 0.4, 1.2), (-1.1, -1.0 / 3.0, -2.0, 1.9), (2.0, 1.0 / 40.0, 3.0, 1.57),
          (0.0, -1.0 / 0.55, 1.0, 0.9), (-4.0, 1.0 / 7.0, -0.3, 2.3)]


def test_exact_helices_give_their_quadruplet_and_parameters():
    geo = geometry_cmslike()
    for (z0, kappa, phi, theta) in TRACKS:
        xyz, lay = _event(geo, [(z0, kappa, phi, theta)])
        r = oracle.seed_quads(geo, xyz, lay, **CUTS)
        assert r["hits"].shape[0] == 1
        assert list(r["hits"][0]) == [0, 1, 2, 3]
        p = r["par"][0]
        assert abs(p[2] - z0) < 1e-9 and abs(p[3] - kappa) < 1e-9 * max(1.0, abs(kappa))
        assert abs(np.remainder(p[4] - phi + np.pi, 2 * np.pi) - np.pi) < 1e-9
        assert abs(p[5] - theta) < 1e-9
        assert p[0] == 0.0 and p[1] == 0.0


def test_curvature_margin_closed_form():
    geo = geometry_cmslike()
    for f in (1.02, 1.5, 4.0):
        xyz, lay = _event(geo, [(0.0, 1.0 / (CUTS["pt_min"] * f), 0.7, 1.4)])
        r = oracle.seed_quads(geo, xyz, lay, **CUTS)
        assert r["hits"].shape[0] == 1
        assert abs(r["margin"][0] - (1.0 - 1.0 / f)) < 1e-9
    xyz, lay = _event(geo, [(0.0, 1.0 / (CUTS["pt_min"] * 0.98), 0.7, 1.4)])
    assert oracle.seed_quads(geo, xyz, lay, **CUTS)["hits"].shape[0] == 0
    r = oracle.seed_quads(geo, xyz, lay, eps=0.05, **CUTS)
    assert abs(r["margin"][0] - (1.0 - 1.0 / 0.98)) < 1e-9


def test_z0_margin_closed_form():
    geo = geometry_cmslike()
    for z0 in (4.9, -4.5, 5.2):
        xyz, lay = _event(geo, [(z0, 1.0 / 20.0, 0.2, 1.3)])   # pT 20: curvature margin 0.975
        r = oracle.seed_quads(geo, xyz, lay, eps=0.1, **CUTS)
        assert r["hits"].shape[0] == 1
        assert abs(r["margin"][0] - (1.0 - abs(z0) / CUTS["z_max"])) < 1e-9


def test_last_layer_residual_margins_closed_form():
    geo = geometry_cmslike()
    ids, radii = oracle.seeding_layers(geo)
    base = (0.0, 1.0 / 20.0, 0.2, 1.3)
    for d in (0.001, -0.002, 0.0035):   # turn the layer-3 hit by d radians about z
        xyz, lay = _event(geo, [base])
        x, y = xyz[3, 0], xyz[3, 1]
        xyz[3, 0], xyz[3, 1] = x * np.cos(d) - y * np.sin(d), x * np.sin(d) + y * np.cos(d)
        r = oracle.seed_quads(geo, xyz, lay, eps=0.2, **CUTS)
        assert abs(r["margin"][0] - (1.0 - radii[3] * abs(np.sin(d)) / CUTS["rphi_tol"])) < 1e-9
    for dz in (0.03, -0.09, 0.11):
        xyz, lay = _event(geo, [base])
        xyz[3, 2] += dz
        r = oracle.seed_quads(geo, xyz, lay, eps=0.2, **CUTS)
        assert abs(r["margin"][0] - (1.0 - abs(dz) / CUTS["z_tol"])) < 1e-9


def test_mirror_images_through_the_beam_line_are_not_seeds():
    """A layer-1 hit on the far side of the beam line defines a nearly straight
    circle through the origin, and a layer-3 hit turned by pi has the same sine
    residual: neither may make a seed."""
    geo = geometry_cmslike()
    base = (0.0, 1.0 / 20.0, 0.2, 1.3)
    for k in (1, 3):
        xyz, lay = _event(geo, [base])
        xyz[k, 0:2] *= -1.0
        assert oracle.seed_quads(geo, xyz, lay, eps=0.5, **CUTS)["hits"].shape[0] == 0, k
    # with both the genuine and the mirrored layer-3 hit only the genuine one is used
    xyz, lay = _event(geo, [base])
    xyz = np.concatenate([xyz, xyz[3:4] * np.array([-1.0, -1.0, 1.0])])
    lay = np.concatenate([lay, lay[3:4]])
    r = oracle.seed_quads(geo, xyz, lay, **CUTS)
    assert [list(h) for h in r["hits"]] == [[0, 1, 2, 3]]


def _noisy_event():
    ev = sev.make_config_event(2, n_tracks=400)
    return ev.geom, ev.hit_xyz, ev.hit_layer


def _key(r):
    return {tuple(h): i for i, h in enumerate(r["hits"])}


def test_symmetries():
    geo, xyz, lay = _noisy_event()
    r0 = oracle.seed_quads(geo, xyz, lay, **CUTS)
    assert r0["hits"].shape[0] > 100
    k0 = _key(r0)
    a = 0.37
    rot = xyz.copy()
    rot[:, 0] = xyz[:, 0] * np.cos(a) - xyz[:, 1] * np.sin(a)
    rot[:, 1] = xyz[:, 0] * np.sin(a) + xyz[:, 1] * np.cos(a)
    mz = xyz * np.array([1.0, 1.0, -1.0])
    my = xyz * np.array([1.0, -1.0, 1.0])
    for name, x2 in (("rot", rot), ("mirror z", mz), ("mirror y", my)):
        r = oracle.seed_quads(geo, x2, lay, **CUTS)
        k = _key(r)
        # margins move by rounding only; compare the quadruplets away from the cuts
        strong0 = {q for q, i in k0.items() if r0["margin"][i] > 1e-9}
        strong = {q for q, i in k.items() if r["margin"][i] > 1e-9}
        assert strong0 == strong, name
        for q in strong0:
            p0, p = r0["par"][k0[q]], r["par"][k[q]]
            dphi = lambda u, v: abs(np.remainder(u - v + np.pi, 2 * np.pi) - np.pi)
            if name == "rot":
                assert abs(p[2] - p0[2]) < 1e-9 and abs(p[3] - p0[3]) < 1e-9 * max(1, abs(p0[3]))
                assert dphi(p[4], p0[4] + a) < 1e-9 and abs(p[5] - p0[5]) < 1e-9
            elif name == "mirror z":
                assert abs(p[2] + p0[2]) < 1e-9 and abs(p[3] - p0[3]) < 1e-9 * max(1, abs(p0[3]))
                assert dphi(p[4], p0[4]) < 1e-9 and abs(p[5] - (np.pi - p0[5])) < 1e-9
            else:
                assert abs(p[2] - p0[2]) < 1e-9 and abs(p[3] + p0[3]) < 1e-9 * max(1, abs(p0[3]))
                assert dphi(p[4], -p0[4]) < 1e-9 and abs(p[5] - p0[5]) < 1e-9


def test_events_are_independent():
    geo, xyz, lay = _noisy_event()
    r1 = oracle.seed_quads(geo, xyz, lay, **CUTS)
    xyz2 = np.concatenate([xyz, xyz]); lay2 = np.concatenate([lay, lay])
    H = lay.shape[0]
    r2 = oracle.seed_quads(geo, xyz2, lay2, np.array([0, H, 2 * H]), **CUTS)
    n = r1["hits"].shape[0]
    assert r2["hits"].shape[0] == 2 * n
    assert np.array_equal(r2["hits"][:n], r1["hits"]) and np.array_equal(r2["hits"][n:], r1["hits"] + H)
    assert np.array_equal(r2["event"], np.repeat([0, 1], n))


def test_needs_four_barrels():
    from synth.geometry import _mk
    g = _mk([(0, 4.0, -10, 10, 0.01, 0.01, 0.01)] * 3 + [(1, 30.0, 4, 16, 0.01, 0.01, 0.01)], 3.8, "x")
    with pytest.raises(ValueError):
        oracle.seeding_layers(g)
