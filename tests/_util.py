"""Helpers shared by the GPU tests: marshal synthetic events to device tensors,
run the CUDA path through the C ABI binding, compare with the oracle."""
import numpy as np
import torch

# discrete decisions whose relative margin is below this are not compared
# exactly (chi2 at the cut, rank ties at the N-th place, acceptance edges)
FRAGILE_TOL = 1e-4
# parameter / covariance agreement (FP32 GPU vs FP64 oracle)
PAR_RTOL = 1e-4
COV_RTOL = 1e-4
# sum of chi2: residuals of ~sigma formed from FP32 positions of ~100 cm carry
# ~1e-4 relative error each, so the chi2 sum is compared at 1e-3 relative
CHI2_RTOL = 1e-3


def f32(a, dev):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)


def i32(a, dev):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.int32, device=dev)


def i64(a, dev):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.int64, device=dev)


def make_ctx(geom, n_phi_bins=64, n_w_bins=16, device=0):
    import paper_2002_06295_gb300 as mkf
    ctx = mkf.Context(device)
    mkf.mkf_load_geometry(ctx, geom.table(), geom.bz, n_phi_bins, n_w_bins)
    return ctx


def gpu_build(ctx, events, *, max_cands, chi2_cut=30.0, max_holes=3, min_hits=4, dup_frac=0.5, debug=False):
    """Bin + build all events in one call; returns numpy outputs."""
    import paper_2002_06295_gb300 as mkf
    dev = torch.device("cuda", ctx.device)
    xyz = np.concatenate([e.hit_xyz for e in events], 0)
    lcov = np.concatenate([e.hit_lcov for e in events], 0)
    layer = np.concatenate([e.hit_layer for e in events], 0)
    hoff = np.concatenate([[0], np.cumsum([e.n_hits for e in events])])
    sp = np.concatenate([e.seed_par for e in events], 0)
    sc = np.concatenate([e.seed_cov for e in events], 0)
    soff = np.concatenate([[0], np.cumsum([e.n_seeds for e in events])])
    mkf.mkf_set_debug(ctx, debug)
    mkf.mkf_bin_hits(ctx, f32(xyz.T, dev), f32(lcov.T, dev), i32(layer, dev), i64(hoff, dev))
    out = mkf.mkf_build_tracks(ctx, f32(sp.T, dev), f32(sc.T, dev), i64(soff, dev), chi2_cut=chi2_cut,
                               max_cands=max_cands, max_holes=max_holes, min_hits=min_hits, dup_frac=dup_frac)
    mkf.mkf_sync(ctx)
    stats = mkf.mkf_get_stats(ctx)
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["par"] = res["par"].T.astype(np.float64)
    res["cov"] = res["cov"].T.astype(np.float64)
    res["nhits"], res["nholes"], res["nsteps"] = res["counts"]
    res["stats"] = stats
    res["hit_off"] = hoff
    res["seed_off"] = soff
    return res


def oracle_build(events, *, max_cands, chi2_cut=30.0, max_holes=3, min_hits=4, dup_frac=0.5, seeds=None,
                 dedup=True):
    """Oracle per event (global hit ids), concatenated."""
    import oracle
    outs = []
    base = 0
    for e in events:
        geo = oracle.Geo.of(e.geom)
        sp, sc = e.seed_par, e.seed_cov
        if seeds is not None:
            sp, sc = sp[seeds], sc[seeds]
        outs.append(oracle.build_event(geo, e.hit_xyz, e.hit_lcov, e.hit_layer, sp, sc, chi2_cut=chi2_cut,
                                       max_cands=max_cands, max_holes=max_holes, min_hits=min_hits,
                                       dup_frac=dup_frac, tol=FRAGILE_TOL, hit_base=base, dedup=dedup))
        base += e.n_hits
    res = {k: np.concatenate([o[k] for o in outs], 0) for k in outs[0] if k != "stats"}
    res["stats"] = {k: sum(o["stats"][k] for o in outs) for k in outs[0]["stats"]}
    return res


def par_rel_err(a, b):
    """|a - b| per parameter relative to max(|b|, 1) (kappa: |b|); phi wrapped."""
    d = np.abs(a - b)
    d[:, 4] = np.abs((a[:, 4] - b[:, 4] + np.pi) % (2 * np.pi) - np.pi)
    den = np.maximum(np.abs(b), 1.0)
    den[:, 3] = np.abs(b[:, 3])
    return d / den


def cov_scales(b):
    """Per-parameter scale of a packed covariance: sqrt(C_ii) for kappa, phi,
    theta; for x, y, z the square root of the largest eigenvalue of the 3x3
    position block (on a surface one position direction has zero variance, so
    its diagonal entry is no scale)."""
    M = np.zeros(b.shape[:-1] + (3, 3))
    for i in range(3):
        for j in range(i + 1):
            M[..., i, j] = M[..., j, i] = b[..., i * (i + 1) // 2 + j]
    lam = np.linalg.eigvalsh(M)[..., -1]
    s = np.zeros(b.shape[:-1] + (6,))
    s[..., :3] = np.sqrt(np.maximum(lam, 0))[..., None]
    for i in range(3, 6):
        s[..., i] = np.sqrt(np.abs(b[..., i * (i + 1) // 2 + i]))
    return s


def cov_rel_err(a, b):
    """|C_a - C_b| / (s_i s_j) over the packed entries, s from cov_scales(b)."""
    s = cov_scales(b)
    out = np.zeros_like(a)
    for i in range(6):
        for j in range(i + 1):
            k = i * (i + 1) // 2 + j
            out[:, k] = np.abs(a[:, k] - b[:, k]) / np.maximum(s[:, i] * s[:, j], 1e-300)
    return out


def compare(gpu, ref, sel=None, fragile_tol=FRAGILE_TOL):
    """Exact comparison of the discrete results on seeds whose decisions are
    not within fragile_tol of flipping; numeric agreement on those that match."""
    n = ref["hits"].shape[0]
    idx = np.arange(n) if sel is None else np.asarray(sel)
    g = {k: (v[idx] if isinstance(v, np.ndarray) and v.shape[:1] == (gpu["hits"].shape[0],) else v)
         for k, v in gpu.items()}
    robust = ref["margin"] >= fragile_tol
    same_hits = (g["hits"] == ref["hits"]).all(1)
    same_layers = (g["layers"] == ref["layers"]).all(1)
    same_counts = (g["nhits"] == ref["nhits"]) & (g["nholes"] == ref["nholes"]) & (g["nsteps"] == ref["nsteps"])
    match = same_hits & same_layers & same_counts
    rep = dict(n=n, robust=int(robust.sum()), fragile=int((~robust).sum()),
               mismatch_robust=int((robust & ~match).sum()), mismatch_fragile=int((~robust & ~match).sum()))
    m = robust & match
    if m.any():
        pe = par_rel_err(g["par"][m], ref["par"][m])
        rep["par_err"] = float(pe.max())
        rep["par_err_per"] = [float(x) for x in pe.max(0)]
        ce = cov_rel_err(g["cov"][m], ref["cov"][m])
        rep["cov_err"] = float(ce.max())
        rep["cov_frac_ok"] = float((ce.max(1) < COV_RTOL).mean())
        w, k = np.unravel_index(np.argmax(ce), ce.shape)
        seed = int(idx[np.nonzero(m)[0][w]])
        rep["cov_worst"] = dict(seed=seed, entry=int(k), gpu=float(g["cov"][m][w, k]), ref=float(ref["cov"][m][w, k]),
                                nsteps=int(ref["nsteps"][np.nonzero(m)[0][w]]),
                                nholes=int(ref["nholes"][np.nonzero(m)[0][w]]))
        rep["score_err"] = float((np.abs(g["score"][m] - ref["score"][m]) / np.maximum(1, np.abs(ref["score"][m]))).max())
    bad = np.nonzero(robust & ~match)[0]
    rep["bad_seeds"] = bad[:10].tolist()
    rep["bad_detail"] = [dict(seed=int(idx[b]), margin=float(ref["margin"][b]),
                              gpu_hits=g["hits"][b][:g["nsteps"][b]].tolist(),
                              ref_hits=ref["hits"][b][:ref["nsteps"][b]].tolist(),
                              gpu_layers=g["layers"][b][:g["nsteps"][b]].tolist(),
                              ref_layers=ref["layers"][b][:ref["nsteps"][b]].tolist(),
                              gpu_score=float(g["score"][b]), ref_score=float(ref["score"][b]))
                         for b in bad[:3]]
    return rep


def cov_ok(ce, frac=0.99, tol=COV_RTOL, cap=1e-3):
    """Covariance agreement where a stated fraction of the results may exceed
    the bar: at least `frac` of the tracks within `tol` (scale metric) and
    none beyond `cap`."""
    per = ce.max(1) if ce.ndim == 2 else ce
    return bool((per < tol).mean() >= frac and per.max() < cap)
