"""FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

Plain, slow reference of the combinatorial Kalman-filter building, of the
fixed-assignment Kalman fit (and its reference gradient), of strip clustering
and of hit-based seeding.  Only ``tests/``,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import it;
the CUDA library never does, and the two share no code.

The arithmetic lives in ``mkf_oracle.cpp`` (scalar C++ templated on the number
type); this module compiles it with g++ on first use and wraps it with ctypes.
"""
import ctypes
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mkf_oracle.cpp")
_SRCS = (_SRC, os.path.join(_HERE, "strip_oracle.cpp"), os.path.join(_HERE, "seed_oracle.cpp"))
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

D = ctypes.POINTER(ctypes.c_double)
I = ctypes.POINTER(ctypes.c_int)
LL = ctypes.POINTER(ctypes.c_longlong)


def build(force=False):
    """Compile the oracle (g++, -O2, no target-specific flags)."""
    arch = _LIB + ".arch"
    arch_ok = os.path.exists(arch) and open(arch).read().strip() == platform.machine()
    if not force and arch_ok and os.path.exists(_LIB) and \
            os.path.getmtime(_LIB) >= max(os.path.getmtime(f) for f in _SRCS):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp] + list(_SRCS))
    os.replace(tmp, _LIB)
    with open(arch, "w") as f:
        f.write(platform.machine())
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            c_int, c_double, c_long = ctypes.c_int, ctypes.c_double, ctypes.c_long
            L.orc_path.argtypes = [D, c_int, c_double, D, c_int, c_int, D, D]
            L.orc_path.restype = c_int
            L.orc_helix.argtypes = [c_double, D, c_double, D]
            L.orc_helix.restype = None
            L.orc_transport.argtypes = [D, c_int, c_double, D, D, c_int, c_int, c_int, D, D, D]
            L.orc_transport.restype = c_int
            L.orc_update.argtypes = [c_int, D, D, D, D, D, D]
            L.orc_update.restype = c_double
            L.orc_next_surface.argtypes = [D, c_int, c_double, D, c_double, c_double, D]
            L.orc_next_surface.restype = c_int
            L.orc_build.argtypes = [D, c_int, c_double, D, D, I, c_int, c_long, D, D, c_int,
                                    c_double, c_int, c_int, c_int, c_double, c_double,
                                    I, I, D, D, D, D, I, I, I, I, I, D, LL, c_int]
            L.orc_build.restype = c_int
            L.orc_dedup.argtypes = [c_int, c_int, I, D, I, c_int, c_double, I]
            L.orc_dedup.restype = c_int
            L.orc_fit.argtypes = [D, c_int, c_double, D, D, I, c_int, I, c_int, D, D, c_int, D, D,
                                  c_int, D, D, D, I]
            L.orc_fit.restype = c_int
            L.orc_fit_grad.argtypes = [D, c_int, c_double, D, D, I, c_int, I, c_int, D, D, c_int,
                                       D, D, D, D, D, D, D, D]
            L.orc_fit_grad.restype = c_int
            P = ctypes.c_void_p
            L.orc_strip_clusters.argtypes = [c_int, c_int, P, P, P, c_int, c_int, c_int, I, I, I, I, D]
            L.orc_strip_clusters.restype = c_int
            L.orc_seed_quads.argtypes = [P, P, ctypes.c_longlong, P, c_int, P, P, c_double, c_double, c_double,
                                         c_double, c_double, c_double, ctypes.c_longlong, P, P, P, P]
            L.orc_seed_quads.restype = ctypes.c_longlong
            L.orc_overlaps.argtypes = [P, c_int, c_double, P, P, P, c_int, P, c_int, P, c_int, P, P, c_int,
                                       c_double, c_double, c_double, P, P, P, P]
            L.orc_overlaps.restype = c_int
            _lib = L
    return _lib


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _pd(a):
    return None if a is None else a.ctypes.data_as(D)


def _pi(a):
    return None if a is None else a.ctypes.data_as(I)


def cov_index(i, j):
    if i < j:
        i, j = j, i
    return i * (i + 1) // 2 + j


def unpack_cov(c21):
    """[..., 21] packed lower triangle -> [..., 6, 6] symmetric."""
    c21 = np.asarray(c21)
    out = np.zeros(c21.shape[:-1] + (6, 6), c21.dtype)
    for i in range(6):
        for j in range(i + 1):
            out[..., i, j] = out[..., j, i] = c21[..., cov_index(i, j)]
    return out


def pack_cov(m):
    m = np.asarray(m)
    out = np.zeros(m.shape[:-2] + (21,), m.dtype)
    for i in range(6):
        for j in range(i + 1):
            out[..., cov_index(i, j)] = m[..., i, j]
    return out


class Geo:
    """Layer table [L,5] (kind, pos, lo, hi, x0) + field, as the oracle wants it."""

    def __init__(self, table, bz):
        self.table = _d(table)
        self.L = int(self.table.shape[0])
        self.bz = float(bz)

    @classmethod
    def of(cls, geom):
        return cls(geom.table(), geom.bz)


def helix(bz, p, s):
    q = np.zeros(6)
    lib().orc_helix(float(bz), _pd(_d(p)), float(s), _pd(q))
    return q


def path(geo, p, layer, direction=+1):
    s = np.zeros(1)
    q = np.zeros(6)
    ok = lib().orc_path(_pd(geo.table), geo.L, geo.bz, _pd(_d(p)), int(layer), int(direction), _pd(s), _pd(q))
    return (float(s[0]), q) if ok else (None, None)


def transport(geo, p, C, layer, direction=+1, material=False):
    """Returns (p', C'[21], J[6,6]) or None when the surface is not crossed."""
    po = np.zeros(6); Co = np.zeros(21); J = np.zeros(36)
    ok = lib().orc_transport(_pd(geo.table), geo.L, geo.bz, _pd(_d(p)), _pd(_d(C)), int(layer),
                             int(direction), int(bool(material)), _pd(po), _pd(Co), _pd(J))
    return (po, Co, J.reshape(6, 6)) if ok else None


def update(kind, p, C, hit_xyz, hit_lcov):
    """Returns (chi2, p', C')."""
    po = np.zeros(6); Co = np.zeros(21)
    chi2 = lib().orc_update(int(kind), _pd(_d(p)), _pd(_d(C)), _pd(_d(hit_xyz)), _pd(_d(hit_lcov)),
                            _pd(po), _pd(Co))
    return chi2, po, Co


def next_surface(geo, p, rho_ref=0.0, zeta_ref=0.0):
    s = np.zeros(1)
    l = lib().orc_next_surface(_pd(geo.table), geo.L, geo.bz, _pd(_d(p)), float(rho_ref),
                               float(zeta_ref), _pd(s))
    return int(l), float(s[0])


def build_event(geo, hit_xyz, hit_lcov, hit_layer, seed_par, seed_cov, *, chi2_cut=30.0, max_cands=4,
                max_holes=3, min_hits=4, dup_frac=0.5, tol=1e-4, hit_base=0, dedup=True):
    """Combinatorial building of one event, brute-force hit search.  Returns a
    dict of per-seed arrays (see orc_build in mkf_oracle.cpp)."""
    hx, hc, hl = _d(hit_xyz), _d(hit_lcov), _i(hit_layer)
    sp, sc = _d(seed_par), _d(seed_cov)
    H, S, L = int(hl.shape[0]), int(sp.shape[0]), geo.L
    out = dict(hits=np.zeros((S, L), np.int32), layers=np.zeros((S, L), np.int32),
               par=np.zeros((S, 6)), cov=np.zeros((S, 21)), score=np.zeros(S), chi2=np.zeros(S),
               nhits=np.zeros(S, np.int32), nholes=np.zeros(S, np.int32), nsteps=np.zeros(S, np.int32),
               flags=np.zeros(S, np.int32), fragile=np.zeros(S, np.int32), margin=np.zeros(S))
    stats = np.zeros(8, np.int64)
    lib().orc_build(_pd(geo.table), L, geo.bz, _pd(hx), _pd(hc), _pi(hl), H, int(hit_base), _pd(sp), _pd(sc), S,
                    float(chi2_cut), int(max_cands), int(max_holes), int(min_hits), float(dup_frac), float(tol),
                    _pi(out["hits"]), _pi(out["layers"]), _pd(out["par"]), _pd(out["cov"]), _pd(out["score"]),
                    _pd(out["chi2"]), _pi(out["nhits"]), _pi(out["nholes"]), _pi(out["nsteps"]),
                    _pi(out["flags"]), _pi(out["fragile"]), _pd(out["margin"]),
                    stats.ctypes.data_as(LL), int(bool(dedup)))
    out["stats"] = dict(cand_steps=int(stats[0]), chi2_evals=int(stats[1]), updates=int(stats[2]))
    return out


def dedup(hits, score, nhits, min_hits=4, dup_frac=0.5):
    h = _i(hits); sc = _d(score); nh = _i(nhits)
    S, L = h.shape
    flags = np.zeros(S, np.int32)
    lib().orc_dedup(int(S), int(L), _pi(h), _pd(sc), _pi(nh), int(min_hits), float(dup_frac), _pi(flags))
    return flags


def fit(geo, hit_xyz, hit_lcov, hit_layer, hits, init_par, init_cov, *, align=None, x0=None, direction=+1):
    """Fixed-assignment fit; returns (par [T,6], cov [T,21], chi2 [T], ok [T])."""
    hx, hc, hl = _d(hit_xyz), _d(hit_lcov), _i(hit_layer)
    h = _i(hits)
    T, K = h.shape
    ip, ic = _d(init_par), _d(init_cov)
    al = None if align is None else _d(align)
    xx = None if x0 is None else _d(x0)
    par = np.zeros((T, 6)); cov = np.zeros((T, 21)); chi2 = np.zeros(T); ok = np.zeros(T, np.int32)
    lib().orc_fit(_pd(geo.table), geo.L, geo.bz, _pd(hx), _pd(hc), _pi(hl), int(hl.shape[0]), _pi(h), int(K),
                  _pd(ip), _pd(ic), int(T), _pd(al), _pd(xx), int(direction), _pd(par), _pd(cov), _pd(chi2),
                  _pi(ok))
    return par, cov, chi2, ok


def fit_grad(geo, hit_xyz, hit_lcov, hit_layer, hits, init_par, init_cov, g_chi2, *, g_par=None, g_cov=None,
             align=None, x0=None):
    """Dual-number gradient of sum_t g_chi2 chi2_t + g_par.p + g_cov.C (packed)
    with respect to hit xyz [H,3], alignment [L,3] and thickness [L]."""
    hx, hc, hl = _d(hit_xyz), _d(hit_lcov), _i(hit_layer)
    h = _i(hits)
    T, K = h.shape
    H = int(hl.shape[0])
    ip, ic = _d(init_par), _d(init_cov)
    al = None if align is None else _d(align)
    xx = None if x0 is None else _d(x0)
    gh = np.zeros((H, 3)); ga = np.zeros((geo.L, 3)); gx = np.zeros(geo.L)
    gp = None if g_par is None else _d(g_par)
    gc = None if g_cov is None else _d(g_cov)
    lib().orc_fit_grad(_pd(geo.table), geo.L, geo.bz, _pd(hx), _pd(hc), _pi(hl), H, _pi(h), int(K), _pd(ip),
                       _pd(ic), int(T), _pd(al), _pd(xx), _pd(_d(g_chi2)), _pd(gp), _pd(gc), _pd(gh), _pd(ga),
                       _pd(gx))
    return gh, ga, gx


def overlaps(geo, hit_xyz, hit_lcov, hit_layer, hits, init_par, init_cov, ev_hit_off=None, chi2_cut=20.0,
             max_drphi=1.0, max_dw=10.0):
    """Overlap-hit recovery (a second hit on the layer of each track hit, in
    the adjacent-module box |d(r phi)| <= max_drphi, |dw| <= max_dw around it,
    best predicted chi2 against the fitted state after that hit, below
    chi2_cut).
    hits [T, K] global ids; init_par [T, 6], init_cov [T, 21].  Returns dict
    hit [T, K] (-1: none), chi2, gap (relative chi2 gap to the runner-up) and
    best (best candidate chi2, passing or not)."""
    hx, hc, hl = _d(hit_xyz), _d(hit_lcov), _i(hit_layer)
    h = _i(hits)
    T, K = h.shape
    H = int(hl.shape[0])
    off = np.ascontiguousarray([0, H] if ev_hit_off is None else ev_hit_off, np.int64)
    ip, ic = _d(init_par), _d(init_cov)
    out = {"hit": np.zeros((T, K), np.int32), "chi2": np.zeros((T, K)), "gap": np.zeros((T, K)),
           "best": np.zeros((T, K))}
    lib().orc_overlaps(geo.table.ctypes.data, geo.L, geo.bz, hx.ctypes.data, hc.ctypes.data, hl.ctypes.data, H,
                       off.ctypes.data, off.size - 1, h.ctypes.data, int(K), ip.ctypes.data, ic.ctypes.data, int(T),
                       float(chi2_cut), float(max_drphi), float(max_dw), out["hit"].ctypes.data,
                       out["chi2"].ctypes.data, out["gap"].ctypes.data,
                       out["best"].ctypes.data)
    return out


def strip_clusters(adc, noise_q, bad, max_bad_gap=1, q_min=30):
    """Strip clustering of Sec. 4 on modules [M, N] (adc, noise_q uint16 with
    noise_q = 8 x noise, bad uint8).  Returns dict of arrays module, first,
    last, charge (int) and center (charge-weighted strip index), in module
    order and, within a module, in strip order."""
    a = np.ascontiguousarray(adc, np.uint16)
    nq = np.ascontiguousarray(noise_q, np.uint16)
    b = np.ascontiguousarray(bad, np.uint8)
    M, N = a.shape
    cap = max(1, M * (N // 2 + 1))
    out = {k: np.zeros(cap, np.int32) for k in ("module", "first", "last", "charge")}
    center = np.zeros(cap)
    n = lib().orc_strip_clusters(int(M), int(N), a.ctypes.data, nq.ctypes.data, b.ctypes.data, int(max_bad_gap),
                                 int(q_min), int(cap), _pi(out["module"]), _pi(out["first"]), _pi(out["last"]),
                                 _pi(out["charge"]), _pd(center))
    res = {k: v[:n].copy() for k, v in out.items()}
    res["center"] = center[:n].copy()
    return res


SEED_LAYERS_NEEDED = 4


def seeding_layers(geo):
    """The four innermost barrel layers (ids, radii), innermost first."""
    kind = np.asarray(geo.kind)
    pos = np.asarray(geo.pos, np.float64)
    ids = [int(i) for i in np.argsort(np.where(kind == 0, pos, np.inf), kind="stable") if kind[i] == 0]
    if len(ids) < SEED_LAYERS_NEEDED:
        raise ValueError("seeding needs four barrel layers")
    ids = ids[:SEED_LAYERS_NEEDED]
    return np.array(ids, np.int32), pos[ids].astype(np.float64)


def seed_quads(geo, hit_xyz, hit_layer, ev_hit_off=None, *, pt_min=0.5, z_max=5.0, rphi_tol=0.05, z_tol=0.1,
               eps=0.0):
    """Hit-based seeding (Sec. 3, four innermost barrel layers, prompt tracks):
    every quadruplet whose smallest cut margin is >= -eps.  hit_xyz [H, 3],
    hit_layer [H]; ev_hit_off [E+1] CSR (default one event).  Returns dict
    hits [n, 4] (global hit ids), margin [n], par [n, 6] at the beam line,
    event [n]."""
    xyz = np.ascontiguousarray(hit_xyz, np.float64)
    lay = np.ascontiguousarray(hit_layer, np.int32)
    H = lay.shape[0]
    off = np.ascontiguousarray([0, H] if ev_hit_off is None else ev_hit_off, np.int64)
    ids, radii = seeding_layers(geo)
    cap = 1 << 16
    while True:
        hits = np.zeros((cap, 4), np.int32)
        marg = np.zeros(cap)
        par = np.zeros((cap, 6))
        ev = np.zeros(cap, np.int32)
        n = lib().orc_seed_quads(xyz.ctypes.data, lay.ctypes.data, H, off.ctypes.data, off.size - 1,
                                 ids.ctypes.data, radii.ctypes.data, float(geo.bz), float(pt_min), float(z_max),
                                 float(rphi_tol), float(z_tol), float(eps), cap, hits.ctypes.data,
                                 marg.ctypes.data, par.ctypes.data, ev.ctypes.data)
        if n <= cap:
            return {"hits": hits[:n].copy(), "margin": marg[:n].copy(), "par": par[:n].copy(),
                    "event": ev[:n].copy()}
        cap = int(n)
