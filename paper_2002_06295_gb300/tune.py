"""Autotuner of the building launch: hit-bin granularity (phi x z|r bins per
layer), warps per block and lanes per seed.  Every candidate is run on the
caller's own event batch and timed with the library's CUDA events (binning +
building); the fastest is applied to the context and cached on disk per
(GPU, geometry, max_cands, workload size class).  Results do not depend on the
choice (the search window is conservative for any binning)."""
import hashlib
import json
import math
import os

import torch

from . import api

BIN_CHOICES = ((32, 8), (64, 16), (128, 16), (128, 32), (256, 32), (256, 64), (256, 128))
WARP_CHOICES = (2, 4, 8)


def _cache_path():
    root = os.environ.get("MKF_CACHE_DIR") or os.path.join(os.path.expanduser("~"), ".cache", "mkf_gb300")
    return os.path.join(root, "autotune.json")


def _key(ctx, table, bz, max_cands, n_seeds, n_hits):
    g = hashlib.sha1(json.dumps([[float(v) for v in row] for row in table] + [float(bz)]).encode()).hexdigest()[:16]
    name = torch.cuda.get_device_name(ctx.device)
    return "%s|%s|N%d|S%d|H%d" % (name, g, int(max_cands), int(math.log2(max(n_seeds, 1))),
                                  int(math.log2(max(n_hits, 1))))


def _load_cache():
    try:
        with open(_cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store_cache(c):
    path = _cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(c, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass


def lane_choices(max_cands):
    g = 1
    while g < max_cands:
        g <<= 1
    out = []
    while g <= 32:
        out.append(g)
        g <<= 1
    return out


def apply(ctx, table, bz, cfg, xyz, lcov, layer, ev_hit_off):
    api.mkf_load_geometry(ctx, table, bz, cfg["n_phi"], cfg["n_w"])
    api.mkf_set_build_config(ctx, cfg["warps"], cfg["lanes"])
    api.mkf_bin_hits(ctx, xyz, lcov, layer, ev_hit_off)


def autotune_build(ctx, table, bz, xyz, lcov, layer, ev_hit_off, seed_par, seed_cov, ev_seed_off, *, max_cands,
                   chi2_cut=30.0, max_holes=3, min_hits=4, dup_frac=0.5, reps=2, use_cache=True):
    """Pick and apply the fastest configuration; returns it as a dict
    (n_phi, n_w, warps, lanes, ms).  The context ends loaded with that
    geometry binning and with the hits binned."""
    n_seeds, n_hits = int(seed_par.shape[1]), int(layer.shape[0])
    key = _key(ctx, table, bz, max_cands, n_seeds, n_hits)
    cache = _load_cache() if use_cache else {}
    if key in cache:
        cfg = cache[key]
        apply(ctx, table, bz, cfg, xyz, lcov, layer, ev_hit_off)
        return dict(cfg, cached=True)
    api.mkf_set_timing(ctx, True)
    out = None
    best = None
    for n_phi, n_w in BIN_CHOICES:
        api.mkf_load_geometry(ctx, table, bz, n_phi, n_w)
        api.mkf_bin_hits(ctx, xyz, lcov, layer, ev_hit_off)
        t_bin = api.mkf_get_timings(ctx)["bin"]
        for warps in WARP_CHOICES:
            for lanes in lane_choices(max_cands):
                api.mkf_set_build_config(ctx, warps, lanes)
                times = []
                for _ in range(reps):
                    out = api.mkf_build_tracks(ctx, seed_par, seed_cov, ev_seed_off, chi2_cut=chi2_cut,
                                               max_cands=max_cands, max_holes=max_holes, min_hits=min_hits,
                                               dup_frac=dup_frac, out=out)
                    times.append(api.mkf_get_timings(ctx)["build"])
                ms = min(times) + t_bin
                if best is None or ms < best["ms"]:
                    best = dict(n_phi=n_phi, n_w=n_w, warps=warps, lanes=lanes, ms=ms)
    api.mkf_sync(ctx)
    apply(ctx, table, bz, best, xyz, lcov, layer, ev_hit_off)
    if use_cache:
        cache[key] = best
        _store_cache(cache)
    return dict(best, cached=False)
