"""Thin Python binding of the C ABI (include/mkf.h): the same entry points, with
torch CUDA tensors marshalled to device pointers.  No arithmetic happens here;
every step of the path runs in libmkf.so."""
import ctypes

import torch

from . import _lib

MKF_OK = 0
ERRORS = {-1: "MKF_ERR_ARG", -2: "MKF_ERR_OOM", -3: "MKF_ERR_CUDA", -4: "MKF_ERR_TIMEOUT", -5: "MKF_ERR_STATE",
          -6: "MKF_ERR_CAPACITY"}
TRK_SHORT, TRK_KEPT, TRK_DUP = 0, 1, 2


class MkfError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


def _ptr(t, dtype=None, name="tensor"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if dtype is not None and t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


class Context:
    """Owns an mkf_ctx (one device, one host thread)."""

    def __init__(self, device=0):
        self.lib = _lib.load()
        h = ctypes.c_void_p()
        rc = self.lib.mkf_create(ctypes.byref(h), int(device))
        if rc != MKF_OK:
            raise MkfError(rc, "mkf_create(%d)" % device)
        self.h = h
        self.device = device
        self.n_layers = 0

    def close(self):
        if getattr(self, "h", None):
            self.lib.mkf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc != MKF_OK:
            msg = self.lib.mkf_last_error(self.h)
            raise MkfError(rc, "%s: %s" % (what, msg.decode() if msg else ""))


def mkf_create(device=0):
    return Context(device)


def mkf_destroy(ctx):
    ctx.close()


def mkf_sync(ctx, stream=None):
    ctx._check(ctx.lib.mkf_sync(ctx.h, _stream(stream)), "mkf_sync")


def mkf_load_geometry(ctx, table, bz, n_phi_bins=64, n_w_bins=16):
    """table: [L, 5] rows (kind, pos, lo, hi, x_over_x0); bin counts per layer
    (scalars or sequences)."""
    L = len(table)
    arr = (_lib.MkfLayer * L)()
    for l, row in enumerate(table):
        nphi = n_phi_bins[l] if hasattr(n_phi_bins, "__len__") else n_phi_bins
        nw = n_w_bins[l] if hasattr(n_w_bins, "__len__") else n_w_bins
        arr[l] = _lib.MkfLayer(int(row[0]), float(row[1]), float(row[2]), float(row[3]), float(row[4]), int(nphi),
                               int(nw))
    ctx._check(ctx.lib.mkf_load_geometry(ctx.h, ctypes.cast(arr, ctypes.c_void_p), L, float(bz)),
               "mkf_load_geometry")
    ctx.n_layers = L


def mkf_bin_hits(ctx, xyz, lcov, layer, ev_hit_off, stream=None):
    H = int(layer.shape[0])
    E = int(ev_hit_off.shape[0]) - 1
    ctx._check(ctx.lib.mkf_bin_hits(ctx.h, _ptr(xyz, torch.float32, "xyz"), _ptr(lcov, torch.float32, "lcov"),
                                    _ptr(layer, torch.int32, "layer"), H, _ptr(ev_hit_off, torch.int64, "ev_hit_off"),
                                    E, _stream(stream)), "mkf_bin_hits")
    ctx.n_hits = H
    ctx.n_events = E


def mkf_bin_hits_masked(ctx, xyz, lcov, layer, ev_hit_off, mask=None, stream=None):
    """mkf_bin_hits leaving out the hits with mask[h] != 0 (uint8 tensor [H])."""
    H = int(layer.shape[0])
    E = int(ev_hit_off.shape[0]) - 1
    ctx._check(ctx.lib.mkf_bin_hits_masked(ctx.h, _ptr(xyz, torch.float32, "xyz"), _ptr(lcov, torch.float32, "lcov"),
                                           _ptr(layer, torch.int32, "layer"), H,
                                           _ptr(ev_hit_off, torch.int64, "ev_hit_off"), E,
                                           _ptr(mask, torch.uint8, "mask"), _stream(stream)), "mkf_bin_hits_masked")
    ctx.n_hits = H
    ctx.n_events = E


def mkf_used_hits(ctx, hits, flags, n_hits, mask=None, stream=None):
    """uint8 mask [n_hits] with 1 at every hit of a kept track (added to `mask` if given)."""
    T, L = int(hits.shape[0]), int(hits.shape[1])
    m = mask if mask is not None else torch.zeros(int(n_hits), dtype=torch.uint8, device=hits.device)
    ctx._check(ctx.lib.mkf_used_hits(ctx.h, _ptr(hits, torch.int32, "hits"), L, _ptr(flags, torch.int32, "flags"), T,
                                     int(n_hits), _ptr(m, torch.uint8, "mask"), _stream(stream)), "mkf_used_hits")
    return m


def mkf_get_binning(ctx, stream=None):
    n = ctypes.c_int64()
    ctx._check(ctx.lib.mkf_get_binning(ctx.h, None, None, ctypes.byref(n), _stream(stream)), "mkf_get_binning")
    dev = torch.device("cuda", ctx.device)
    perm = torch.empty(ctx.n_hits, dtype=torch.int32, device=dev)
    off = torch.empty(n.value + 1, dtype=torch.int32, device=dev)
    ctx._check(ctx.lib.mkf_get_binning(ctx.h, _ptr(perm), _ptr(off), ctypes.byref(n), _stream(stream)),
               "mkf_get_binning")
    return perm, off


def alloc_build_outputs(ctx, S, device=None):
    dev = torch.device("cuda", ctx.device) if device is None else device
    L = ctx.n_layers
    return dict(hits=torch.empty((S, L), dtype=torch.int32, device=dev),
                layers=torch.empty((S, L), dtype=torch.int32, device=dev),
                par=torch.empty((6, S), dtype=torch.float32, device=dev),
                cov=torch.empty((21, S), dtype=torch.float32, device=dev),
                score=torch.empty(S, dtype=torch.float32, device=dev),
                chi2=torch.empty(S, dtype=torch.float32, device=dev),
                counts=torch.empty((3, S), dtype=torch.int32, device=dev),
                flags=torch.empty(S, dtype=torch.int32, device=dev))


def mkf_build_tracks(ctx, seed_par, seed_cov, ev_seed_off, chi2_cut=30.0, max_cands=4, max_holes=3, min_hits=4,
                     dup_frac=0.5, out=None, stream=None):
    S = int(seed_par.shape[1])
    o = alloc_build_outputs(ctx, S) if out is None else out
    ctx._check(ctx.lib.mkf_build_tracks(
        ctx.h, _ptr(seed_par, torch.float32, "seed_par"), _ptr(seed_cov, torch.float32, "seed_cov"),
        _ptr(ev_seed_off, torch.int64, "ev_seed_off"), S, float(chi2_cut), int(max_cands), int(max_holes),
        int(min_hits), float(dup_frac), _ptr(o["hits"]), _ptr(o.get("layers")), _ptr(o["par"]), _ptr(o["cov"]),
        _ptr(o["score"]), _ptr(o["chi2"]), _ptr(o.get("counts")), _ptr(o["flags"]), _stream(stream)),
        "mkf_build_tracks")
    return o


def mkf_set_build_config(ctx, warps_per_block=4, lanes_per_seed=0):
    ctx._check(ctx.lib.mkf_set_build_config(ctx.h, int(warps_per_block), int(lanes_per_seed)), "mkf_set_build_config")


def mkf_set_build_dedup(ctx, enabled=True):
    ctx._check(ctx.lib.mkf_set_build_dedup(ctx.h, int(enabled)), "mkf_set_build_dedup")


def mkf_set_adjoint_config(ctx, lanes_per_track=0):
    ctx._check(ctx.lib.mkf_set_adjoint_config(ctx.h, int(lanes_per_track)), "mkf_set_adjoint_config")


STRIP_SPLITS = ((32, 1, 1), (32, 1, 2), (32, 1, 3), (32, 1, 4), (32, 2, 2), (64, 1, 2), (64, 1, 3), (64, 2, 2))


def mkf_set_strip_config(ctx, chunk=0, events_per_item=0, stages=0):
    ctx._check(ctx.lib.mkf_set_strip_config(ctx.h, int(chunk), int(events_per_item), int(stages)),
               "mkf_set_strip_config")


def mkf_set_debug(ctx, brute_force_window_check):
    ctx._check(ctx.lib.mkf_set_debug(ctx.h, int(bool(brute_force_window_check))), "mkf_set_debug")


STAT_NAMES = ("cand_steps", "chi2_evals", "updates", "tracks_kept", "window_violations", "nav_tests", "seeds",
              "chi2_full")


def mkf_get_stats(ctx, stream=None):
    buf = (ctypes.c_int64 * 8)()
    ctx._check(ctx.lib.mkf_get_stats(ctx.h, ctypes.cast(buf, ctypes.c_void_p), len(STAT_NAMES), _stream(stream)), "mkf_get_stats")
    return {k: int(buf[i]) for i, k in enumerate(STAT_NAMES)}


TIMER_NAMES = ("build", "bin", "dedup", "fit", "adjoint", "backward")


def mkf_set_timing(ctx, on=True):
    ctx._check(ctx.lib.mkf_set_timing(ctx.h, int(bool(on))), "mkf_set_timing")


def mkf_get_timings(ctx, stream=None):
    """Device milliseconds of the most recent call of each stage (-1: not run)."""
    buf = (ctypes.c_float * 8)()
    ctx._check(ctx.lib.mkf_get_timings(ctx.h, ctypes.cast(buf, ctypes.c_void_p), 6, _stream(stream)),
               "mkf_get_timings")
    return {k: float(buf[i]) for i, k in enumerate(TIMER_NAMES)}


def mkf_cluster_strips(ctx, adc, noise_q, bad, max_bad_gap=1, q_min=30, max_out=None, out=None, stream=None):
    """Strip clustering of adc [E*M, N] (uint16) with noise_q [M, N] (uint16) and
    bad [M, N] (uint8).  Returns dict row, first, last, charge, center (device
    tensors of max_out entries, unordered) and count (device int64 [1])."""
    R, N = int(adc.shape[0]), int(adc.shape[1])
    M = int(noise_q.shape[0])
    if R % M:
        raise ValueError("adc rows must be a multiple of the module count")
    dev = adc.device
    cap = int(max_out) if max_out is not None else max(1, R * N // 8)
    o = out or dict(row=torch.empty(cap, dtype=torch.int32, device=dev),
                    first=torch.empty(cap, dtype=torch.int32, device=dev),
                    last=torch.empty(cap, dtype=torch.int32, device=dev),
                    charge=torch.empty(cap, dtype=torch.int32, device=dev),
                    center=torch.empty(cap, dtype=torch.float32, device=dev),
                    count=torch.zeros(1, dtype=torch.int64, device=dev))
    cap = int(o["row"].shape[0])
    ctx._check(ctx.lib.mkf_cluster_strips(ctx.h, _ptr(adc, torch.uint16, "adc"), _ptr(noise_q, torch.uint16, "noise_q"),
                                          _ptr(bad, torch.uint8, "bad"), R // M, M, N, int(max_bad_gap), int(q_min),
                                          _ptr(o["row"]), _ptr(o["first"]), _ptr(o["last"]), _ptr(o["charge"]),
                                          _ptr(o["center"]), cap, _ptr(o["count"], torch.int64, "count"),
                                          _stream(stream)), "mkf_cluster_strips")
    return o


def mkf_set_seed_config(ctx, max_triplets=0):
    ctx._check(ctx.lib.mkf_set_seed_config(ctx.h, int(max_triplets)), "mkf_set_seed_config")


def mkf_seed_tracks(ctx, pt_min=0.5, z_max=5.0, rphi_tol=0.05, z_tol=0.1, max_seeds=None, out=None, stream=None,
                    read_count=True):
    """Hit-based seeding (four innermost barrel layers) from the binned hits.
    Returns dict par [6, n], cov [21, n] (views ready for mkf_build_tracks),
    hits [n, 4], ev_seed_off [E+1] (device int64) and n (read back, one
    synchronising copy).  With read_count=False (for a fixed triplet capacity,
    mkf_set_seed_config, e.g. inside a CUDA graph) nothing is read back: n is
    None and par [6, max_seeds], cov [21, max_seeds], hits [max_seeds, 4] are
    the whole buffers, in the column stride max_seeds the call then uses."""
    dev = torch.device("cuda", ctx.device)
    cap = int(max_seeds) if max_seeds is not None else max(1024, int(ctx.n_hits))
    E = int(ctx.n_events)
    o = out or dict(par=torch.empty(6 * cap, dtype=torch.float32, device=dev),
                    cov=torch.empty(21 * cap, dtype=torch.float32, device=dev),
                    hits=torch.empty(4 * cap, dtype=torch.int32, device=dev),
                    ev_seed_off=torch.empty(E + 1, dtype=torch.int64, device=dev))
    cap = int(o["hits"].numel()) // 4
    ctx._check(ctx.lib.mkf_seed_tracks(ctx.h, float(pt_min), float(z_max), float(rphi_tol), float(z_tol), cap,
                                       _ptr(o["par"]), _ptr(o["cov"]), _ptr(o["hits"]),
                                       _ptr(o["ev_seed_off"], torch.int64, "ev_seed_off"), _stream(stream)),
               "mkf_seed_tracks")
    res = dict(o)
    if not read_count:
        res["n"] = None
        res["par"] = o["par"].view(6, cap)
        res["cov"] = o["cov"].view(21, cap)
        res["hits"] = o["hits"].view(cap, 4)
        return res
    n = int(o["ev_seed_off"][E].item())
    res["n"] = n
    if n <= cap:
        res["par"] = o["par"][:6 * n].view(6, n)
        res["cov"] = o["cov"][:21 * n].view(21, n)
        res["hits"] = o["hits"][:4 * n].view(n, 4)
    return res


def mkf_find_overlaps(ctx, xyz, lcov, layer, hits, init_par, init_cov, chi2_cut=20.0, max_drphi=1.0, max_dw=10.0,
                      out=None, stream=None):
    """Overlap hits of tracks (hits [T, K] int32, init_par [6, T], init_cov
    [21, T]); xyz, lcov, layer as for mkf_bin_hits (the binned hits).
    Returns dict hit [T, K] int32 (-1: none) and chi2 [T, K] (device)."""
    T, K = int(hits.shape[0]), int(hits.shape[1])
    H = int(layer.shape[0])
    dev = hits.device
    o = out or dict(hit=torch.empty((T, K), dtype=torch.int32, device=dev),
                    chi2=torch.empty((T, K), dtype=torch.float32, device=dev))
    ctx._check(ctx.lib.mkf_find_overlaps(ctx.h, _ptr(xyz, torch.float32, "xyz"), _ptr(lcov, torch.float32, "lcov"),
                                         _ptr(layer, torch.int32, "layer"), H, _ptr(hits, torch.int32, "hits"), K,
                                         _ptr(init_par, torch.float32, "init_par"),
                                         _ptr(init_cov, torch.float32, "init_cov"), T, float(chi2_cut),
                                         float(max_drphi), float(max_dw), _ptr(o["hit"]), _ptr(o["chi2"]),
                                         _stream(stream)), "mkf_find_overlaps")
    return o


OVERLAP_STAT_NAMES = ("hits_fitted", "candidates", "found")


def mkf_set_overlap_config(ctx, lanes_per_track=0):
    ctx._check(ctx.lib.mkf_set_overlap_config(ctx.h, int(lanes_per_track)), "mkf_set_overlap_config")


def mkf_get_overlap_stats(ctx, stream=None):
    buf = (ctypes.c_int64 * len(OVERLAP_STAT_NAMES))()
    ctx._check(ctx.lib.mkf_get_overlap_stats(ctx.h, ctypes.cast(buf, ctypes.c_void_p), len(OVERLAP_STAT_NAMES),
                                             _stream(stream)), "mkf_get_overlap_stats")
    return {k: int(buf[i]) for i, k in enumerate(OVERLAP_STAT_NAMES)}


SEED_STAT_NAMES = ("l1_examined", "pairs", "l2_examined", "triplets", "l3_examined", "seeds")


def mkf_get_seed_stats(ctx, stream=None):
    buf = (ctypes.c_int64 * len(SEED_STAT_NAMES))()
    ctx._check(ctx.lib.mkf_get_seed_stats(ctx.h, ctypes.cast(buf, ctypes.c_void_p), len(SEED_STAT_NAMES),
                                          _stream(stream)), "mkf_get_seed_stats")
    return {k: int(buf[i]) for i, k in enumerate(SEED_STAT_NAMES)}


def mkf_dedup_tracks(ctx, hits, score, nhits, ev_seed_off, n_hits_total, min_hits=4, dup_frac=0.5, out_flags=None,
                     stream=None):
    S, L = int(hits.shape[0]), int(hits.shape[1])
    E = int(ev_seed_off.shape[0]) - 1
    flags = torch.empty(S, dtype=torch.int32, device=hits.device) if out_flags is None else out_flags
    ctx._check(ctx.lib.mkf_dedup_tracks(ctx.h, _ptr(hits, torch.int32, "hits"), L, _ptr(score, torch.float32),
                                        _ptr(nhits, torch.int32), _ptr(ev_seed_off, torch.int64), E, S,
                                        int(n_hits_total), int(min_hits), float(dup_frac), _ptr(flags),
                                        _stream(stream)), "mkf_dedup_tracks")
    return flags


def mkf_dedup_tracks_noalloc(hits, score, nhits, ev_seed_off, n_hits_total, min_hits=4, dup_frac=0.5,
                             out_flags=None, out_status=None, stream=None):
    """Duplicate removal that allocates no device memory inside the library
    (fixed working array; see include/mkf.h for its limits).  Returns the
    status code; flags and status are written to the given device tensors."""
    S, L = int(hits.shape[0]), int(hits.shape[1])
    E = int(ev_seed_off.shape[0]) - 1
    return _lib.load().mkf_dedup_tracks_noalloc(
        _ptr(hits, torch.int32, "hits"), L, _ptr(score, torch.float32, "score"), _ptr(nhits, torch.int32, "nhits"),
        _ptr(ev_seed_off, torch.int64, "ev_seed_off"), E, S, int(n_hits_total), int(min_hits), float(dup_frac),
        _ptr(out_flags, torch.int32, "out_flags"), _ptr(out_status, torch.int32, "out_status"), _stream(stream))


def mkf_fit_tracks(ctx, xyz, lcov, layer, hits, init_par, init_cov, align=None, x0=None, ckpt=None, out=None,
                   stream=None):
    H = int(layer.shape[0])
    T, K = int(hits.shape[0]), int(hits.shape[1])
    dev = xyz.device
    o = out or dict(par=torch.empty((6, T), dtype=torch.float32, device=dev),
                    cov=torch.empty((21, T), dtype=torch.float32, device=dev),
                    chi2=torch.empty(T, dtype=torch.float32, device=dev),
                    ok=torch.empty(T, dtype=torch.int32, device=dev))
    ctx._check(ctx.lib.mkf_fit_tracks(ctx.h, _ptr(xyz, torch.float32, "xyz"), _ptr(lcov, torch.float32, "lcov"),
                                      _ptr(layer, torch.int32, "layer"), H, _ptr(hits, torch.int32, "hits"), K,
                                      _ptr(init_par, torch.float32), _ptr(init_cov, torch.float32), T,
                                      _ptr(align, torch.float32), _ptr(x0, torch.float32), _ptr(o["par"]),
                                      _ptr(o["cov"]), _ptr(o["chi2"]), _ptr(o["ok"]), _ptr(ckpt, torch.float32),
                                      _stream(stream)), "mkf_fit_tracks")
    return o


def mkf_fit_backward(ctx, xyz, lcov, layer, hits, init_par, align=None, x0=None, out=None, stream=None):
    H = int(layer.shape[0])
    T, K = int(hits.shape[0]), int(hits.shape[1])
    dev = xyz.device
    o = out or dict(par=torch.empty((6, T), dtype=torch.float32, device=dev),
                    cov=torch.empty((21, T), dtype=torch.float32, device=dev),
                    chi2=torch.empty(T, dtype=torch.float32, device=dev),
                    ok=torch.empty(T, dtype=torch.int32, device=dev))
    ctx._check(ctx.lib.mkf_fit_backward(ctx.h, _ptr(xyz, torch.float32, "xyz"), _ptr(lcov, torch.float32, "lcov"),
                                        _ptr(layer, torch.int32, "layer"), H, _ptr(hits, torch.int32, "hits"), K,
                                        _ptr(init_par, torch.float32), T, _ptr(align, torch.float32),
                                        _ptr(x0, torch.float32), _ptr(o["par"]), _ptr(o["cov"]), _ptr(o["chi2"]),
                                        _ptr(o["ok"]), _stream(stream)), "mkf_fit_backward")
    return o


def mkf_fit_tracks_adjoint(ctx, xyz, lcov, layer, hits, init_par, init_cov, ckpt, g_chi2=None, g_par=None,
                           g_cov=None, align=None, x0=None, out=None, stream=None):
    H = int(layer.shape[0])
    T, K = int(hits.shape[0]), int(hits.shape[1])
    dev = xyz.device
    o = out or dict(g_hit=torch.empty((3, H), dtype=torch.float32, device=dev),
                    g_align=torch.empty((ctx.n_layers, 3), dtype=torch.float32, device=dev),
                    g_x0=torch.empty(ctx.n_layers, dtype=torch.float32, device=dev))
    ctx._check(ctx.lib.mkf_fit_tracks_adjoint(
        ctx.h, _ptr(xyz, torch.float32, "xyz"), _ptr(lcov, torch.float32, "lcov"), _ptr(layer, torch.int32, "layer"),
        H, _ptr(hits, torch.int32, "hits"), K, _ptr(init_par, torch.float32), _ptr(init_cov, torch.float32), T,
        _ptr(align, torch.float32), _ptr(x0, torch.float32), _ptr(ckpt, torch.float32), _ptr(g_chi2, torch.float32),
        _ptr(g_par, torch.float32), _ptr(g_cov, torch.float32), _ptr(o["g_hit"]), _ptr(o["g_align"]),
        _ptr(o["g_x0"]), _stream(stream)), "mkf_fit_tracks_adjoint")
    return o
