#!/usr/bin/env python
"""Throughput benchmark of the Kalman-filter track-building path on one GB300.

One step = the whole path on one CMS-like event (38 surfaces, 5000 tracks,
~85k hits with 20 % noise, 6 candidates per seed): hit binning -> combinatorial
building with duplicate removal -> forward fit of every found track (with
per-layer checkpoints) -> adjoint of that fit -> backward fit.  Inputs are
synthetic (seeded), generated on the host and resident in HBM before the timed
region; the L2 is flushed between timed steps (inputs are smaller than L2).

Metric: candidate Kalman steps per second (one step = one candidate
propagated to one surface with all its chi2 evaluations and its update),
counted by the kernel itself; events/s and fitted tracks/s are reported beside.

Multi-GPU (torchrun): events are independent, each rank builds its own event
(weak scaling), no collective on the data path; the max over ranks of the
timed region is reported.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "c1": "C1 event: 10-cylinder barrel, 100 tracks, 4 candidates/seed, chi2<30, then refit (fwd + adjoint + bwd) "
          "of every found track",
    "c2": "C2 CMS-like event: 38 surfaces (14 barrel + 24 disk), 5000 tracks, ~85k hits incl. 20% noise, "
          "6 candidates/seed, chi2<30, then refit (fwd + adjoint + bwd) of every found track",
    "c3": "C3 batch: 256 events of the 10-cylinder barrel, 200..8000 tracks/event, 4 candidates/seed, "
          "then refit (fwd + adjoint + bwd) of every found track",
    "c5": "C5 batch: 64 events x 10000 tracks, 10-cylinder barrel, 50% noise, 8 candidates/seed, "
          "then refit (fwd + adjoint + bwd) of every found track"}
METRIC = "candidate Kalman steps/s"
UNIT = "cand-steps/s"

# FP32 work per unit, counted from the kernel formulas as executed (FMA = 2,
# add/mul/div = 1; sqrt, rsqrt, sin/cos, atan, log not counted); barrel-surface
# counts, so disk-heavy work is under-counted
FLOPS_NAV_TEST = 44       # one surface whose crossing the navigation computed (crossing path + acceptance)
# one candidate step: helix 46 + Jacobian 84 + material 25 + window ~35 + the
# U-D transport 676 (J U rows 120, the theta row 17, Gram-Schmidt of rows 4..0
# 455, position covariance 84)
FLOPS_CAND_STEP = 866
FLOPS_BOX = 7             # one candidate-hit pair examined: residuals r_a, r_b + half-plane test
FLOPS_CHI2 = 33           # rest of the chi2 of a pair that passes the box test (with the Cauchy-Schwarz floor)
# one Kalman update of a kept child: two Bierman scalar updates (140 each) and
# the hit covariance's decorrelation, rows and residuals (21)
FLOPS_UPDATE = 301
FP32_LANES = 128          # per SM (Blackwell)
# FP32 work per track-hit of the fit gradient (C4), counted the same way: the
# outward U-D fit step (path 41, helix 46, Jacobian 84, material 25, U-D
# transport 676, update 301, checkpoint C = U D U^T 189, cot and omega 2), and
# the adjoint step with its recompute (path, helix, Jacobian 171, plain
# J C J^T 408, material 27, update quantities 138), the update reverse 718,
# the transport reverse 846, six material dual passes (~80 each) and seven
# propagation dual passes (path, helix and Jacobian on dual numbers, an add
# costing 2, a multiply 4 and an FMA 6 flops: ~3 x 171, plus the contraction
# 56), and the hit-frame terms 20
FLOPS_FIT_HIT = 1364
FLOPS_ADJ_HIT = 6795
# HBM bytes per track-hit of the fit gradient: the 27-float checkpoint written
# by the fit and read by the adjoint, the hit's xyz, covariance and layer read
# by both, its slot of the hit list read by both; per track: seed state read
# by both, fit outputs written; per hit: its gradient written
BYTES_FIT_TRACKHIT = 2 * 108 + 2 * 28 + 2 * 4
BYTES_FIT_TRACK = 2 * 108 + 116
BYTES_FIT_HIT = 12
# HBM bytes of the binning stage: per hit, its xyz, covariance and layer read
# twice (key pass, scatter pass), its key and rank written and read, two
# 32-byte records written; per bin, the count written and read by the scan
# and the offset written
BYTES_BIN_HIT = 2 * 28 + 2 * 8 + 2 * 32
BYTES_BIN_BIN = 12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="mkf", choices=["mkf", "reference"])
    ap.add_argument("--cpu-sample-seeds", type=int, default=0,
                    help="seeds per oracle sample (0: sized for ~15 s of CPU work)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true", help="skip the C3 batched-vs-plain and C4 fit-gradient lines")
    ap.add_argument("--workload", default="c2", choices=["c2", "c3", "c5"],
                    help="timed workload (c2: the CMS-like event the metric is quoted on)")
    ap.add_argument("--no-graph", action="store_true", help="time eager launches only (no CUDA-graph replay)")
    ap.add_argument("--only", choices=["strips", "seeding", "overlaps", "in_flight", "fit_gradient"],
                    help="run one secondary measurement alone and print it (for profiling its kernel)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# oracle (CPU) timing: used by the cpu_baseline field and by --impl reference
_EV = None


def _worker_init():
    global _EV
    sys.path.insert(0, ROOT)
    import synth
    _EV = synth.make_config_event(2)


def _worker_build(seeds):
    import oracle
    import numpy as np
    ev = _EV
    t0 = time.perf_counter()
    out = oracle.build_event(oracle.Geo.of(ev.geom), ev.hit_xyz, ev.hit_lcov, ev.hit_layer, ev.seed_par[seeds],
                             ev.seed_cov[seeds], chi2_cut=30.0, max_cands=6, max_holes=3, min_hits=4, dup_frac=0.5,
                             dedup=False)
    return out["stats"]["cand_steps"], time.perf_counter() - t0, int(np.asarray(seeds).size)


def oracle_pool(n_workers):
    import multiprocessing as mp
    import oracle
    oracle.build()   # compile once before the workers load it
    ctx = mp.get_context("spawn")
    return ctx.Pool(n_workers, initializer=_worker_init)


def oracle_step(pool, n_workers, n_seeds, offset):
    """Oracle building of n_seeds seeds of the event (spread over the pool)."""
    import numpy as np
    seeds = (offset + np.arange(n_seeds)) % 5000
    chunks = [c for c in np.array_split(seeds, n_workers) if c.size]
    t0 = time.perf_counter()
    res = pool.map(_worker_build, chunks)
    dt = time.perf_counter() - t0
    return sum(r[0] for r in res), dt


def n_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_reference(args):
    """The reference arm: the FP64 oracle as it stands, on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = n_cores()
    pool = oracle_pool(cores)
    per_step = args.cpu_sample_seeds or 24 * cores
    for w in range(args.warmup):
        oracle_step(pool, cores, max(cores, per_step // 4), 1000 * w)
    units = 0
    elapsed = 0.0
    for k in range(args.steps):
        u, dt = oracle_step(pool, cores, per_step, 97 * k)
        units += u
        elapsed += dt
    pool.close()
    value = units / elapsed
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "C2 CMS-like event: 38 surfaces (14 barrel + 24 disk), 5000 tracks, ~85k hits "
                                   "incl. 20% noise, 6 candidates/seed, chi2<30; building only (the oracle has no "
                                   "refit at this scale: its gradient takes one dual-number pass per input)",
                       "sample": "%d seeds of the event per step" % per_step},
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d seeds x %d steps of the 5000-seed event, brute-force hit search, "
                                       "one process per core" % (per_step, args.steps)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measure_batched(mkf, tune, dev, reps=3):
    """C3: 256 events of uneven size (200..8000 tracks, log-uniform) built in
    one call (batched, persistent kernel) against 256 single-event calls of
    the same library (plain).  Device time of binning + building + dedup."""
    import torch

    import synth
    b = synth.make_batch(3)
    g = b.geom
    spec = synth.WORKLOAD_SPECS[3]
    kw = dict(chi2_cut=spec["chi2_cut"], max_cands=spec["max_cands"], max_holes=spec["max_holes"],
              min_hits=spec["min_hits"], dup_frac=spec["dup_frac"])
    f32 = dict(dtype=torch.float32, device=dev)
    xyz = torch.tensor(b.cat("hit_xyz").T.copy(), **f32)
    lcov = torch.tensor(b.cat("hit_lcov").T.copy(), **f32)
    lay = torch.tensor(b.cat("hit_layer"), dtype=torch.int32, device=dev)
    sp = torch.tensor(b.cat("seed_par").T.copy(), **f32)
    sc = torch.tensor(b.cat("seed_cov").T.copy(), **f32)
    hoff = torch.tensor(b.hit_off, dtype=torch.int64, device=dev)
    soff = torch.tensor(b.seed_off, dtype=torch.int64, device=dev)
    ctx = mkf.Context(dev.index)
    mkf.mkf_load_geometry(ctx, g.table(), g.bz)
    tb = tune.autotune_build(ctx, g.table(), g.bz, xyz, lcov, lay, hoff, sp, sc, soff, max_cands=kw["max_cands"])
    out = None
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, device=dev)
    bt = []
    for r in range(reps + 1):
        flush.fill_(float(r))
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        mkf.mkf_bin_hits(ctx, xyz, lcov, lay, hoff)
        out = mkf.mkf_build_tracks(ctx, sp, sc, soff, out=out, **kw)
        e.record(stream)
        e.synchronize()
        if r:
            bt.append(a.elapsed_time(e))
    steps = mkf.mkf_get_stats(ctx)["cand_steps"]
    # plain: the same library called once per event (configuration tuned on one event)
    evs = []
    for i, ev in enumerate(b.events):
        evs.append(dict(xyz=torch.tensor(ev.hit_xyz.T.copy(), **f32), lcov=torch.tensor(ev.hit_lcov.T.copy(), **f32),
                        lay=torch.tensor(ev.hit_layer, dtype=torch.int32, device=dev),
                        hoff=torch.tensor([0, ev.n_hits], dtype=torch.int64, device=dev),
                        sp=torch.tensor(ev.seed_par.T.copy(), **f32), sc=torch.tensor(ev.seed_cov.T.copy(), **f32),
                        soff=torch.tensor([0, ev.n_seeds], dtype=torch.int64, device=dev)))
    big = max(range(len(evs)), key=lambda i: b.events[i].n_seeds)
    e0 = evs[big]
    tp = tune.autotune_build(ctx, g.table(), g.bz, e0["xyz"], e0["lcov"], e0["lay"], e0["hoff"], e0["sp"], e0["sc"],
                             e0["soff"], max_cands=kw["max_cands"])
    outs = [mkf.alloc_build_outputs(ctx, b.events[i].n_seeds) for i in range(len(evs))]

    def plain():
        for i, x in enumerate(evs):
            mkf.mkf_bin_hits(ctx, x["xyz"], x["lcov"], x["lay"], x["hoff"])
            mkf.mkf_build_tracks(ctx, x["sp"], x["sc"], x["soff"], out=outs[i], **kw)

    pt = []
    for r in range(2):
        flush.fill_(float(r))
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        plain()
        e.record(stream)
        e.synchronize()
        pt.append(a.elapsed_time(e))
    mkf.mkf_sync(ctx)
    # the plain sequence of 256 x (bin + build + dedup) launched as one CUDA graph
    pg_ms = None
    try:
        mkf.mkf_set_timing(ctx, False)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            plain()
        g.replay()
        torch.cuda.synchronize()
        pg = []
        for r in range(2):
            flush.fill_(float(r))
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            g.replay()
            e.record(stream)
            e.synchronize()
            pg.append(a.elapsed_time(e))
        pg_ms = min(pg)
    except Exception:
        pg_ms = None
    mkf.mkf_set_timing(ctx, True)
    mkf.mkf_sync(ctx)
    ctx.close()
    E = b.n_events
    bms, pms = min(bt), min(pt)
    return {"workload": "C3: 256 events of the 10-cylinder barrel, 200..8000 tracks/event (log-uniform), "
                        "%d seeds, %d hits, 4 candidates/seed" % (int(b.seed_off[-1]), int(b.hit_off[-1])),
            "batched_ms": bms, "plain_ms": pms, "batched_events_per_s": E / (bms * 1e-3),
            "plain_events_per_s": E / (pms * 1e-3), "batched_over_plain": pms / bms,
            "plain_graph_ms": pg_ms, "batched_over_plain_graph": None if pg_ms is None else pg_ms / bms,
            "batched_cand_steps_per_s": steps / (bms * 1e-3),
            "tuned_batched": {k: tb[k] for k in ("n_phi", "n_w", "warps", "lanes")},
            "tuned_plain": {k: tp[k] for k in ("n_phi", "n_w", "warps", "lanes")}}


def measure_in_flight(mkf, dev, counts=(1, 2, 4), rounds=20):
    """C2 events in flight: S distinct C2 events (event seeds 0..S-1), each
    with its own context, stream and captured CUDA graph of the whole step
    (binning -> building -> dedup -> forward fit -> adjoint beside the inward
    fit), started together after an L2 flush; a round ends when all S are
    done.  The step and the events are those of the C2 headline; only the
    number of events on the GPU at once changes (the paper's throughput runs
    likewise give each thread its own event)."""
    import numpy as np
    import torch

    import synth
    from paper_2002_06295_gb300 import tune
    spec = synth.WORKLOAD_SPECS[2]
    kw = dict(chi2_cut=spec["chi2_cut"], max_cands=spec["max_cands"], max_holes=spec["max_holes"],
              min_hits=spec["min_hits"], dup_frac=spec["dup_frac"])

    def make(e):
        ev = synth.make_config_event(2, e)
        g = ev.geom
        ctx = mkf.Context(dev.index)
        mkf.mkf_load_geometry(ctx, g.table(), g.bz, 64, 16)
        t = lambda a, dt=torch.float32: torch.tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
        d = dict(xyz=t(ev.hit_xyz.T), lcov=t(ev.hit_lcov.T), layer=t(ev.hit_layer, torch.int32),
                 hoff=t([0, ev.n_hits], torch.int64), sp=t(ev.seed_par.T), sc=t(ev.seed_cov.T),
                 soff=t([0, ev.n_seeds], torch.int64))
        tune.autotune_build(ctx, g.table(), g.bz, d["xyz"], d["lcov"], d["layer"], d["hoff"], d["sp"], d["sc"],
                            d["soff"], **kw)
        S, L = ev.n_seeds, g.n_layers
        out = mkf.alloc_build_outputs(ctx, S)
        ckpt = torch.empty((L, 27, S), device=dev)
        res = lambda: dict(par=torch.empty((6, S), device=dev), cov=torch.empty((21, S), device=dev),
                           chi2=torch.empty(S, device=dev), ok=torch.empty(S, dtype=torch.int32, device=dev))
        fit_out, bwd_out = res(), res()
        g_chi2 = torch.ones(S, device=dev)
        adj = dict(g_hit=torch.empty((3, ev.n_hits), device=dev), g_align=torch.empty((L, 3), device=dev),
                   g_x0=torch.empty(L, device=dev))
        main = torch.cuda.Stream(device=dev)
        step_d = make_step(mkf, ctx, kw, ev.n_hits, out, ckpt, fit_out, bwd_out, adj, g_chi2)
        step = lambda: step_d(d)

        with torch.cuda.stream(main):
            for _ in range(3):
                step()
        torch.cuda.synchronize()
        mkf.mkf_sync(ctx)
        units = mkf.mkf_get_stats(ctx)["cand_steps"]   # counters of the last build call
        cg = torch.cuda.CUDAGraph()
        with torch.cuda.stream(main):
            with torch.cuda.graph(cg, stream=main):
                step()
        torch.cuda.synchronize()
        return dict(ctx=ctx, graph=cg, stream=main, units=units, keep=(d, out, ckpt, fit_out, bwd_out, adj, step_d))

    items = [make(e) for e in range(max(counts))]
    flush = torch.empty(256 * 1024 * 1024 // 4, device=dev)   # > 129 MB L2
    base = torch.cuda.current_stream()
    per = {}
    for n in counts:
        its = items[:n]
        for _ in range(3):
            for it in its:
                with torch.cuda.stream(it["stream"]):
                    it["graph"].replay()
        torch.cuda.synchronize()
        times = []
        for r in range(rounds):
            flush.fill_(float(r))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(base)
            ends = []
            for it in its:
                it["stream"].wait_event(a)
                with torch.cuda.stream(it["stream"]):
                    it["graph"].replay()
                e = torch.cuda.Event()
                e.record(it["stream"])
                ends.append(e)
            for e in ends:
                base.wait_event(e)
            b.record(base)
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b))
        units = sum(it["units"] for it in its)
        total = sum(times)
        per[str(n)] = {"ms_per_round": total / rounds, "ms_per_event": total / rounds / n,
                       "value": units * rounds / (total * 1e-3), "events_per_s": n * rounds / (total * 1e-3),
                       "gpu_launches": LAUNCHES_PER_STEP * n * rounds}
    for it in items:
        it["graph"] = None
        it["ctx"].close()
    return {"workload": "C2 step, S distinct C2 events in flight (one context, stream and CUDA graph each)",
            "unit": UNIT, "l2": "flushed (256 MB write) between rounds", "rounds": rounds, "by_events_in_flight": per}


def measure_fit_gradient(mkf, dev, reps=3):
    """C4: 100k tracks with fixed 14-hit assignments on the 14-cylinder barrel:
    outward fit with per-layer checkpoints + hand-written adjoint of sum chi2."""
    import numpy as np
    import torch

    import synth
    g = synth.geometry_barrel14()
    rng = np.random.default_rng(synth.config_seed(4))
    ev = synth.simulate_event(g, 100000, rng, pt_range=(1.0, 10.0), eta_max=0.8)
    hits = ev.true_hits[(ev.true_hits >= 0).sum(1) == 14]
    keep = (ev.true_hits >= 0).sum(1) == 14
    T, K = hits.shape
    f32 = dict(dtype=torch.float32, device=dev)
    xyz = torch.tensor(ev.hit_xyz.T.copy(), **f32)
    lcov = torch.tensor(ev.hit_lcov.T.copy(), **f32)
    lay = torch.tensor(ev.hit_layer, dtype=torch.int32, device=dev)
    hd = torch.tensor(hits, dtype=torch.int32, device=dev)
    sp = torch.tensor(ev.seed_par[keep].T.copy(), **f32)
    sc = torch.tensor(ev.seed_cov[keep].T.copy(), **f32)
    ctx = mkf.Context(dev.index)
    mkf.mkf_load_geometry(ctx, g.table(), g.bz)
    ckpt = torch.empty((K, 27, T), **f32)
    gchi = torch.ones(T, **f32)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, device=dev)
    fo = go = None
    ts = []
    for r in range(reps + 1):
        flush.fill_(float(r))
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fo = mkf.mkf_fit_tracks(ctx, xyz, lcov, lay, hd, sp, sc, ckpt=ckpt, out=fo)
        go = mkf.mkf_fit_tracks_adjoint(ctx, xyz, lcov, lay, hd, sp, sc, ckpt, g_chi2=gchi, out=go)
        e.record(stream)
        e.synchronize()
        if r:
            ts.append(a.elapsed_time(e))
    mkf.mkf_sync(ctx)
    ctx.close()
    ms = min(ts)
    n_th = int((hits >= 0).sum())
    flops = n_th * (FLOPS_FIT_HIT + FLOPS_ADJ_HIT)
    byts = n_th * BYTES_FIT_TRACKHIT + T * BYTES_FIT_TRACK + ev.n_hits * BYTES_FIT_HIT
    peak, hbm = fp32_peak(dev), measured_peaks().get("hbm_gbs", 6800.0)
    achieved = flops / (ms * 1e-3) / 1e12
    return {"workload": "C4: %d tracks x 14 hits, barrel of 14 cylinders; outward fit with checkpoints "
                        "(%.0f MB) + adjoint to hit xyz, alignment, thickness" % (T, K * 27 * T * 4 / 1e6),
            "ms": ms, "fit_gradient_tracks_per_s": T / (ms * 1e-3),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                         "algorithmic_flops": flops, "peak_basis": FP32_PEAK_BASIS,
                         "hbm": {"algorithmic_bytes": byts, "achieved_gbs": byts / (ms * 1e-3) / 1e9,
                                 "frac": byts / (ms * 1e-3) / 1e9 / hbm,
                                 "peak_basis": "MEASURED_PEAKS.json hbm_gbs (measured copy)"}}}


def measure_strips(mkf, dev, reps=5):
    """Strip clustering (Sec. 4) over 16 events of a CMS-sized strip tracker
    (15000 modules x 768 strips; 4 distinct synthetic events, each used 4
    times): device time of the clustering kernel, HBM roofline, and the
    oracle on one event on one core."""
    import numpy as np
    import torch

    import oracle
    import synth.strips as strips
    rng = np.random.default_rng(20026)
    M, N, E = 15000, 768, 16
    nq, bad = strips.make_strip_calibration(M, N, rng)
    evs = [strips.make_strip_event(nq, rng) for _ in range(4)]
    adc = torch.from_numpy(np.concatenate([evs[e % 4] for e in range(E)], 0)).to(dev)
    nq_d, bad_d = torch.from_numpy(nq).to(dev), torch.from_numpy(bad).to(dev)
    ctx = mkf.Context(dev.index)
    out = mkf.mkf_cluster_strips(ctx, adc, nq_d, bad_d, max_out=4 << 20)
    stream = torch.cuda.current_stream()
    ts = []
    for r in range(reps + 1):
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        mkf.mkf_cluster_strips(ctx, adc, nq_d, bad_d, out=out)
        e.record(stream)
        e.synchronize()
        if r:
            ts.append(a.elapsed_time(e))
    mkf.mkf_sync(ctx)
    n = int(out["count"].item())
    ctx.close()
    ms = min(ts)
    byts = adc.numel() * 2 + nq.size * 2 + bad.size + n * 20   # ADC stream, calibration once, clusters out
    t0 = time.perf_counter()
    ref = oracle.strip_clusters(evs[0], nq, bad)
    cpu_s = time.perf_counter() - t0
    hbm = measured_peaks().get("hbm_gbs", 6800.0)
    return {"workload": "16 events x 15000 modules x 768 strips (184 M strips, 368 MB of ADC), ~1 % occupancy",
            "ms": ms, "events_per_s": E / (ms * 1e-3), "strips_per_s": E * M * N / (ms * 1e-3),
            "clusters": n, "clusters_per_event_oracle": int(ref["module"].size),
            "roofline": {"bound": "hbm", "achieved": byts / (ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                         "frac": byts / (ms * 1e-3) / 1e9 / hbm, "algorithmic_bytes": byts,
                         "traffic": profiled_traffic("k_strip_cluster", STRIP_SOURCES),
                         "peak_basis": "MEASURED_PEAKS.json hbm_gbs (measured copy)"},
            "cpu_baseline": {"value": M * N / cpu_s, "unit": "strips/s", "cores": 1, "kind": "oracle",
                             "sample": "one event (11.5 M strips)"}}


# Hit-based seeding: FP32 operations per counted step, read from the kernels in
# csrc/seeds.cu (FMA = 2, add/mul/div/sqrt/transcendental call = 1).
FLOPS_SEED_L1 = 40      # a layer-1 hit tested against a layer-0 hit: circle, curvature and z0 cuts
FLOPS_SEED_PAIR = 59    # a passing pair: cuts again plus the layer-2 prediction
FLOPS_SEED_L2 = 10      # a layer-2 hit tested against a prediction (side, r-phi and z residuals)
FLOPS_SEED_TRIP = 58    # a triplet: circle through the origin, layer-0 and layer-2 hits, layer-3 prediction
FLOPS_SEED_L3 = 10      # a layer-3 hit tested against a prediction
FLOPS_SEED_SEED = 45    # a seed: final circle and state


def measure_seeding(mkf, dev, reps=5):
    """Hit-based seeding (four innermost barrel layers) on the C3 batch (256
    events, 5.5 M hits): device time of mkf_seed_tracks (seeding grid, pairs ->
    triplets, triplets -> seeds), its work counters, the FP32 roofline of that
    work, and the oracle on one event on one core."""
    import numpy as np
    import torch

    import oracle
    import synth.events as sev
    cuts = dict(pt_min=0.5, z_max=5.0, rphi_tol=0.15, z_tol=0.3)
    b = sev.make_batch(3)
    xyz, lay, lcov = b.cat("hit_xyz"), b.cat("hit_layer"), b.cat("hit_lcov")
    ctx = mkf.Context(dev.index)
    mkf.mkf_load_geometry(ctx, b.geom.table(), b.geom.bz, 64, 16)
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(dev, dt)
    mkf.mkf_bin_hits(ctx, t(xyz.T, torch.float32), t(lcov.T, torch.float32), t(lay, torch.int32),
                     t(b.hit_off, torch.int64))
    out = mkf.mkf_seed_tracks(ctx, max_seeds=4 << 20, **cuts)
    stream = torch.cuda.current_stream()
    ts = []
    for r in range(reps + 1):
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        o = mkf.mkf_seed_tracks(ctx, out=out, **cuts)
        e.record(stream)
        e.synchronize()
        if r:
            ts.append(a.elapsed_time(e))
    mkf.mkf_sync(ctx)
    w = mkf.mkf_get_seed_stats(ctx)
    peak = fp32_peak(dev)
    # the seeded path as one CUDA graph: binning, seeding with a fixed triplet
    # capacity (no read-back), building the seeds found (count read on the
    # device), outward fit of the built tracks
    graph_ms = None
    try:
        cap = int(o["hits"].numel()) // 4
        mkf.mkf_set_seed_config(ctx, 4 * int(b.hit_off[-1]))
        X, Lc, Ly, O = (t(xyz.T, torch.float32), t(lcov.T, torch.float32), t(lay, torch.int32),
                        t(b.hit_off, torch.int64))
        sbuf = dict(par=torch.zeros(6 * cap, device=dev), cov=torch.zeros(21 * cap, device=dev),
                    hits=torch.zeros(4 * cap, dtype=torch.int32, device=dev),
                    ev_seed_off=torch.zeros(b.n_events + 1, dtype=torch.int64, device=dev))
        bout = mkf.alloc_build_outputs(ctx, cap)
        fout = dict(par=torch.empty((6, cap), device=dev), cov=torch.empty((21, cap), device=dev),
                    chi2=torch.empty(cap, device=dev), ok=torch.empty(cap, dtype=torch.int32, device=dev))
        bkw = dict(chi2_cut=30.0, max_cands=4, max_holes=3, min_hits=4, dup_frac=0.5)

        def seeded_step():
            mkf.mkf_bin_hits(ctx, X, Lc, Ly, O)
            sd = mkf.mkf_seed_tracks(ctx, out=sbuf, read_count=False, **cuts)
            mkf.mkf_build_tracks(ctx, sd["par"], sd["cov"], sd["ev_seed_off"], out=bout, **bkw)
            mkf.mkf_fit_tracks(ctx, X, Lc, Ly, bout["hits"], sd["par"], sd["cov"], out=fout)

        seeded_step()
        torch.cuda.synchronize()
        mkf.mkf_sync(ctx)
        mkf.mkf_set_timing(ctx, False)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            seeded_step()
        gts = []
        for r in range(reps + 1):
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            graph.replay()
            e.record(stream)
            e.synchronize()
            if r:
                gts.append(a.elapsed_time(e))
        mkf.mkf_sync(ctx)
        graph_ms = min(gts)
    except Exception as exc:   # reported, not fatal to the other lines
        graph_ms = "%s: %s" % (type(exc).__name__, str(exc).splitlines()[0][:160])
    ctx.close()
    ms = min(ts)
    flops = (w["l1_examined"] * FLOPS_SEED_L1 + w["pairs"] * FLOPS_SEED_PAIR + w["l2_examined"] * FLOPS_SEED_L2
             + w["triplets"] * FLOPS_SEED_TRIP + w["l3_examined"] * FLOPS_SEED_L3 + w["seeds"] * FLOPS_SEED_SEED)
    ach = flops / (ms * 1e-3) / 1e12
    ev0 = b.events[0]
    t0 = time.perf_counter()
    ref = oracle.seed_quads(ev0.geom, ev0.hit_xyz, ev0.hit_layer, **cuts)
    cpu_s = time.perf_counter() - t0
    return {"workload": "C3: 256 events of the 10-cylinder barrel, %d hits, %d true tracks; cuts %s"
                        % (int(b.hit_off[-1]), int(b.seed_off[-1]), cuts),
            "ms": ms, "events_per_s": b.n_events / (ms * 1e-3), "seeds": int(o["n"]),
            "seeded_build_fit_graph_ms": graph_ms,
            "seeded_build_fit_graph_events_per_s": (b.n_events / (graph_ms * 1e-3)
                                                    if isinstance(graph_ms, float) else None),
            "seeds_per_s": o["n"] / (ms * 1e-3), "work": w,
            "roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                         "frac": ach / peak,
                         "traffic": profiled_traffic("k_seed_triplets", SEED_SOURCES),
                         "peak_basis": FP32_PEAK_BASIS},
            "cpu_baseline": {"value": ev0.n_hits / cpu_s, "unit": "hits/s", "cores": 1, "kind": "oracle",
                             "sample": "event 0 (%d hits, brute force over all layer-0 x layer-1 pairs)"
                                       % ev0.n_hits,
                             "gpu_hits_per_s": int(b.hit_off[-1]) / (ms * 1e-3),
                             "oracle_seeds": int(ref["hits"].shape[0])}}


def measure_overlaps(mkf, dev, reps=5):
    """Overlap-hit recovery on the C2 event with overlapping modules (30 % of
    barrel crossings leave a second hit): build, then time mkf_find_overlaps
    over the built tracks; recovery against the simulation's truth; FP32
    roofline of its work (the fit steps and chi2 of the building kernel's
    formulas); the oracle on a sample of tracks on one core."""
    import numpy as np
    import torch

    import oracle
    import synth.events as sev
    ev = sev.make_config_event(2, overlap_frac=0.3)
    ctx = mkf.Context(dev.index)
    mkf.mkf_load_geometry(ctx, ev.geom.table(), ev.geom.bz, 64, 16)
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(dev, dt)
    xyz, lcov, lay = t(ev.hit_xyz.T, torch.float32), t(ev.hit_lcov.T, torch.float32), t(ev.hit_layer, torch.int32)
    mkf.mkf_bin_hits(ctx, xyz, lcov, lay, t(np.array([0, ev.n_hits]), torch.int64))
    sp, sc = t(ev.seed_par.T, torch.float32), t(ev.seed_cov.T, torch.float32)
    b = mkf.mkf_build_tracks(ctx, sp, sc, t(np.array([0, ev.n_seeds]), torch.int64), chi2_cut=30.0, max_cands=6,
                             max_holes=3, min_hits=4, dup_frac=0.5)
    o = mkf.mkf_find_overlaps(ctx, xyz, lcov, lay, b["hits"], sp, sc)
    stream = torch.cuda.current_stream()
    ts = []
    for r in range(reps + 1):
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        mkf.mkf_find_overlaps(ctx, xyz, lcov, lay, b["hits"], sp, sc, out=o)
        e.record(stream)
        e.synchronize()
        if r:
            ts.append(a.elapsed_time(e))
    mkf.mkf_sync(ctx)
    w = mkf.mkf_get_overlap_stats(ctx)
    peak = fp32_peak(dev)
    bh, flags, gh = b["hits"].cpu().numpy(), b["flags"].cpu().numpy(), o["hit"].cpu().numpy()
    ctx.close()
    ok = tot = 0
    for tr in np.nonzero(flags == mkf.TRK_KEPT)[0]:
        truth = {int(h): k for k, h in enumerate(ev.true_hits[tr]) if h >= 0}
        for k, h in enumerate(bh[tr]):
            if h >= 0 and int(h) in truth and ev.true_overlap[tr, truth[int(h)]] >= 0:
                tot += 1
                ok += gh[tr, k] == ev.true_overlap[tr, truth[int(h)]]
    ms = min(ts)
    flops = w["hits_fitted"] * (FLOPS_CAND_STEP + FLOPS_UPDATE) + w["candidates"] * (FLOPS_BOX + FLOPS_CHI2)
    ach = flops / (ms * 1e-3) / 1e12
    n_s = 500
    t0 = time.perf_counter()
    oracle.overlaps(oracle.Geo.of(ev.geom), ev.hit_xyz, ev.hit_lcov, ev.hit_layer, bh[:n_s], ev.seed_par[:n_s],
                    ev.seed_cov[:n_s])
    cpu_s = time.perf_counter() - t0
    return {"workload": "C2 event with overlapping modules (30 %% of barrel crossings leave a second hit): %d hits, "
                        "%d built tracks; chi2 < 20, box 1 cm (r phi) x 10 cm" % (ev.n_hits, ev.n_seeds),
            "ms": ms, "tracks_per_s": ev.n_seeds / (ms * 1e-3), "work": w,
            "recovered_true_overlaps": ok / tot if tot else None, "true_overlaps_on_kept_tracks": tot,
            "roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                         "frac": ach / peak,
                         "traffic": profiled_traffic("k_overlaps", OVERLAP_SOURCES),
                         "peak_basis": FP32_PEAK_BASIS},
            "cpu_baseline": {"value": n_s / cpu_s, "unit": "tracks/s", "cores": 1, "kind": "oracle",
                             "sample": "the first %d built tracks (brute force over the layer's hits)" % n_s}}


KERNEL_SOURCES = ("paper_2002_06295_gb300/csrc/build.cu", "paper_2002_06295_gb300/csrc/mkf_device.cuh",
                  "paper_2002_06295_gb300/csrc/mkf_ud.cuh", "paper_2002_06295_gb300/csrc/mkf_geom.h")
STRIP_SOURCES = ("paper_2002_06295_gb300/csrc/strips.cu", "paper_2002_06295_gb300/csrc/mkf_geom.h")
SEED_SOURCES = ("paper_2002_06295_gb300/csrc/seeds.cu", "paper_2002_06295_gb300/csrc/mkf_device.cuh",
                "paper_2002_06295_gb300/csrc/mkf_geom.h")
OVERLAP_SOURCES = ("paper_2002_06295_gb300/csrc/overlaps.cu", "paper_2002_06295_gb300/csrc/mkf_device.cuh",
                   "paper_2002_06295_gb300/csrc/mkf_fit_common.cuh", "paper_2002_06295_gb300/csrc/mkf_geom.h")


def kernel_digest(sources=KERNEL_SOURCES):
    """sha1 over a kernel's sources: a profile's counters apply only to the
    kernel they were taken on."""
    import hashlib
    h = hashlib.sha1()
    for f in sources:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def profiled_traffic(name, sources=KERNEL_SOURCES):
    """DRAM bytes (read + write) per launch of a kernel from the ncu summary
    profiles/<name>_ncu.md, or None when the summary is missing or was taken
    on other kernel sources."""
    path = os.path.join(ROOT, "profiles", "%s_ncu.md" % name)
    try:
        with open(path) as f:
            lines = f.read().splitlines()
    except OSError:
        return None
    kv = {}
    for ln in lines:
        if ln.startswith("kernel-source-sha1:") or ln.startswith("dram-bytes-per-launch:"):
            k, v = ln.split(":", 1)
            kv[k] = v.strip()
    if kv.get("kernel-source-sha1") != kernel_digest(sources) or "dram-bytes-per-launch" not in kv:
        return None
    return int(kv["dram-bytes-per-launch"])


def rank_reduce(dist, dev, values, op):
    """Reduce a list of numbers over the ranks ("max", "min" or "sum"); the
    identity on one rank.  Used for the slowest rank's times, the total work of
    all ranks and decisions every rank must take alike."""
    if not dist:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op={"max": dist.ReduceOp.MAX, "min": dist.ReduceOp.MIN, "sum": dist.ReduceOp.SUM}[op])
    return [float(x) for x in t.tolist()]


FP32_PEAK_BASIS = "FP32: SMs x 128 lanes x 2 flop x maximum SM clock (MEASURED_PEAKS.json sm_max_mhz)"


def fp32_peak(dev, max_mhz=None):
    """FP32 CUDA-core peak in TFLOP/s: every SM's 128 FP32 lanes issuing one FMA
    (2 flop) per clock at the maximum SM clock."""
    import torch
    props = torch.cuda.get_device_properties(dev)
    mhz = max_mhz or measured_peaks().get("sm_max_mhz", 2070.0)
    return props.multi_processor_count * FP32_LANES * 2 * mhz * 1e6 / 1e12


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def shard_range(n_total, rank, world):
    """Contiguous range [start, end) of events 0..n_total-1 for one rank: the
    first n_total % world ranks take one event more.  Events are independent
    (Sec. 2: events are processed in parallel), so the ranks need no exchange
    while they build."""
    base, extra = divmod(n_total, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def workload_events(synth, cfg_id, rank=0, world=1):
    """The events of one timed step of a workload on one rank.  Weak scaling:
    the global event sequence of a step holds world x n_events events (a
    workload's n_events per rank) and each rank takes its contiguous range."""
    n = synth.WORKLOAD_SPECS[cfg_id]["n_events"]
    start, end = shard_range(n * world, rank, world)
    return [synth.make_config_event(cfg_id, e) for e in range(start, end)]


def gather_results(dist, local):
    """Rank 0 receives every rank's results in rank order (a host-side gather of
    the ranks' tracks, the only exchange event sharding needs); other ranks
    get None.  The identity on one rank."""
    if not dist:
        return [local]
    out = [None] * dist.get_world_size() if dist.get_rank() == 0 else None
    dist.gather_object(local, out, dst=0)
    return out


def packed(tensors, device, pin=False):
    """One contiguous buffer holding copies of the given tensors, each piece
    starting on a 256-byte boundary, and views of it in their shapes and
    dtypes: the end-to-end path moves its inputs and its results with one copy
    each instead of one per tensor."""
    import torch
    offs, total = {}, 0
    for k, v in tensors.items():
        offs[k] = total
        total += (v.numel() * v.element_size() + 255) // 256 * 256
    buf = torch.empty(max(total, 256), dtype=torch.uint8, device=device, pin_memory=pin)
    views = {}
    for k, v in tensors.items():
        n = v.numel() * v.element_size()
        views[k] = buf[offs[k]:offs[k] + n].view(v.dtype).view(v.shape)
        views[k].copy_(v)
    return buf, views


def make_step(mkf, ctx, kw, n_hits, out, ckpt, fit_out, bwd_out, adj_out, g_chi2):
    """One step of the path as stream-ordered library calls, capturable as one
    CUDA graph: binning -> building -> forward fit with checkpoints -> adjoint
    on the current stream; duplicate removal on a second stream beside the
    fits (it writes only the flags, which no fit reads) and the inward fit on a
    third once the forward fit is done; the current stream waits for both.
    Duplicate removal is switched out of mkf_build_tracks on this context."""
    import torch
    dev = torch.device("cuda", ctx.device)
    mkf.mkf_set_build_dedup(ctx, False)
    dd_side, bwd_side = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    built, dd_done, fwd_done, bwd_done = (torch.cuda.Event() for _ in range(4))

    def step(inp):
        cur = torch.cuda.current_stream()
        mkf.mkf_bin_hits(ctx, inp["xyz"], inp["lcov"], inp["layer"], inp["hoff"])
        mkf.mkf_build_tracks(ctx, inp["sp"], inp["sc"], inp["soff"], out=out, **kw)
        built.record(cur)
        dd_side.wait_event(built)
        mkf.mkf_dedup_tracks(ctx, out["hits"], out["score"], out["counts"][0], inp["soff"], n_hits,
                             min_hits=kw["min_hits"], dup_frac=kw["dup_frac"], out_flags=out["flags"], stream=dd_side)
        dd_done.record(dd_side)
        mkf.mkf_fit_tracks(ctx, inp["xyz"], inp["lcov"], inp["layer"], out["hits"], inp["sp"], inp["sc"],
                           ckpt=ckpt, out=fit_out)
        fwd_done.record(cur)
        bwd_side.wait_event(fwd_done)
        mkf.mkf_fit_backward(ctx, inp["xyz"], inp["lcov"], inp["layer"], out["hits"], fit_out["par"], out=bwd_out,
                             stream=bwd_side)
        bwd_done.record(bwd_side)
        mkf.mkf_fit_tracks_adjoint(ctx, inp["xyz"], inp["lcov"], inp["layer"], out["hits"], inp["sp"], inp["sc"],
                                   ckpt, g_chi2=g_chi2, out=adj_out)
        cur.wait_event(bwd_done)
        cur.wait_event(dd_done)

    return step


def time_path(mkf, dev, evs, spec, steps, warmup, dist=None, clocks=None, graph=True):
    """Time the whole path on one batch of events: binning -> building with
    duplicate removal -> forward fit with checkpoints -> adjoint, beside the
    inward fit on a side stream.  Inputs are resident in HBM before the timed
    region; the L2 is flushed between steps.  The step is timed eagerly and as
    one replayed CUDA graph, and end to end (pinned host inputs copied in,
    results copied out, inside the timed region).  Times are the slowest
    rank's; work counters are summed over the ranks."""
    import numpy as np
    import torch
    from paper_2002_06295_gb300 import tune
    g = evs[0].geom
    ctx = mkf.Context(dev.index)
    mkf.mkf_load_geometry(ctx, g.table(), g.bz, 64, 16)
    f32 = dict(dtype=torch.float32)
    cat = lambda name: np.concatenate([getattr(e, name) for e in evs], 0)
    n_hits = int(sum(e.n_hits for e in evs))
    host = dict(xyz=torch.tensor(cat("hit_xyz").T.copy(), **f32), lcov=torch.tensor(cat("hit_lcov").T.copy(), **f32),
                layer=torch.tensor(cat("hit_layer"), dtype=torch.int32),
                hoff=torch.tensor(np.concatenate([[0], np.cumsum([e.n_hits for e in evs])]), dtype=torch.int64),
                sp=torch.tensor(cat("seed_par").T.copy(), **f32), sc=torch.tensor(cat("seed_cov").T.copy(), **f32),
                soff=torch.tensor(np.concatenate([[0], np.cumsum([e.n_seeds for e in evs])]), dtype=torch.int64))
    hbuf, host = packed(host, "cpu", pin=True)   # pinned host inputs, one buffer
    d = {k: v.to(dev) for k, v in host.items()}
    # launch shape and bin granularity picked on these events (not timed)
    tuned = tune.autotune_build(ctx, g.table(), g.bz, d["xyz"], d["lcov"], d["layer"], d["hoff"], d["sp"], d["sc"],
                                d["soff"], max_cands=spec["max_cands"], chi2_cut=spec["chi2_cut"],
                                max_holes=spec["max_holes"], min_hits=spec["min_hits"], dup_frac=spec["dup_frac"])
    S, L = int(sum(e.n_seeds for e in evs)), g.n_layers
    out = mkf.alloc_build_outputs(ctx, S)
    ckpt = torch.empty((L, 27, S), dtype=torch.float32, device=dev)
    fit_out = dict(par=torch.empty((6, S), device=dev), cov=torch.empty((21, S), device=dev),
                   chi2=torch.empty(S, device=dev), ok=torch.empty(S, dtype=torch.int32, device=dev))
    # the results the end-to-end path reads back live in one device buffer
    rbuf, rv = packed(dict(hits=out["hits"], flags=out["flags"], par=fit_out["par"], chi2=fit_out["chi2"]), dev)
    out["hits"], out["flags"], fit_out["par"], fit_out["chi2"] = rv["hits"], rv["flags"], rv["par"], rv["chi2"]
    bwd_out = dict(par=torch.empty((6, S), device=dev), cov=torch.empty((21, S), device=dev),
                   chi2=torch.empty(S, device=dev), ok=torch.empty(S, dtype=torch.int32, device=dev))
    g_chi2 = torch.ones(S, device=dev)
    adj_out = dict(g_hit=torch.empty((3, n_hits), device=dev), g_align=torch.empty((L, 3), device=dev),
                   g_x0=torch.empty(L, device=dev))
    stream = torch.cuda.current_stream()
    mkf.mkf_set_timing(ctx, True)
    kw = {k: spec[k] for k in ("chi2_cut", "max_cands", "max_holes", "min_hits", "dup_frac")}
    step = make_step(mkf, ctx, kw, n_hits, out, ckpt, fit_out, bwd_out, adj_out, g_chi2)

    ddbuf, dd_inputs = packed(d, dev)   # device copies of the host inputs (e2e), one buffer
    for _ in range(max(warmup, 3)):
        step(d)
    torch.cuda.synchronize()
    mkf.mkf_sync(ctx)
    stats = mkf.mkf_get_stats(ctx)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > 129 MB L2

    if clocks:
        clocks.start()
        time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    tev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    tm_keys = ("build", "bin", "fit", "adjoint", "backward", "dedup")
    stage = {k: [] for k in tm_keys}
    for k in range(steps):
        flush.fill_(float(k))
        tev[k][0].record(stream)
        step(d)
        tev[k][1].record(stream)
        tm = mkf.mkf_get_timings(ctx)
        for key in tm_keys:
            stage[key].append(tm[key])
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    eager_ms = sum(a.elapsed_time(b) for a, b in tev)

    # the same step captured once as a CUDA graph (the library's calls are
    # stream-ordered and allocate nothing once warm) and replayed
    graphs, graph_ms, graph_note = {}, None, None
    if graph:
        mkf.mkf_set_timing(ctx, False)
        try:
            for name, inp in (("dev", d), ("e2e", dd_inputs)):
                cg = torch.cuda.CUDAGraph()
                with torch.cuda.graph(cg):
                    step(inp)
                graphs[name] = cg
            for _ in range(3):
                graphs["dev"].replay()
            torch.cuda.synchronize()
        except Exception as exc:   # capture refused: eager numbers stand
            graphs, graph_note = {}, "%s: %s" % (type(exc).__name__, str(exc).splitlines()[0][:160])
        ok = int(rank_reduce(dist, dev, [1 if graphs else 0], "min")[0])   # replay only if every rank captured
        if ok:
            if dist:
                dist.barrier()
            gev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            for k in range(steps):
                flush.fill_(float(k))
                gev[k][0].record(stream)
                graphs["dev"].replay()
                gev[k][1].record(stream)
            torch.cuda.synchronize()
            if dist:
                dist.barrier()
            graph_ms = sum(a.elapsed_time(b) for a, b in gev)
        else:
            graphs = {}
        mkf.mkf_set_timing(ctx, True)
        mkf.mkf_sync(ctx)
    clk = clocks.stop() if clocks else None
    # every rank takes the slowest rank's times and the same launch mode
    eager_ms, gm = rank_reduce(dist, dev, [eager_ms, graph_ms if graph_ms is not None else float("inf")], "max")
    graph_ms = gm if gm < float("inf") else None
    use_graph = graph_ms is not None and graph_ms < eager_ms
    total_ms = graph_ms if use_graph else eager_ms

    # end to end through the API with host buffers: H2D inputs, path, D2H results
    rhbuf = torch.empty(rbuf.numel(), dtype=torch.uint8, pin_memory=True)
    h2d, d2h = hbuf.numel(), rhbuf.numel()   # bytes of the two copies (pieces padded to 256 bytes)
    e2e_ms = []
    for k in range(steps):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ddbuf.copy_(hbuf, non_blocking=True)
        if use_graph:
            graphs["e2e"].replay()
        else:
            step(dd_inputs)
        rhbuf.copy_(rbuf, non_blocking=True)
        b.record(stream)
        b.synchronize()
        e2e_ms.append(a.elapsed_time(b))
    mkf.mkf_sync(ctx)
    units = rank_reduce(dist, dev, [stats["cand_steps"]], "sum")[0]
    e2e_total = rank_reduce(dist, dev, [sum(e2e_ms)], "max")[0]
    graphs.clear()
    ctx.close()
    return dict(steps=steps, units=units, stats=stats, total_ms=total_ms, eager_ms=eager_ms, graph_ms=graph_ms,
                graph_note=graph_note, use_graph=use_graph, e2e_total_ms=e2e_total, h2d=h2d, d2h=d2h,
                stage={k: statistics.mean(v) for k, v in stage.items()}, n_events=len(evs), S=S, n_hits=n_hits,
                L=L, max_cands=spec["max_cands"], tuned={k: tuned[k] for k in ("n_phi", "n_w", "warps", "lanes")},
                clocks=clk)


# kernels of one step: binning 5 (keys, 3-pass scan, scatter), building 2
# (seed order, build), dedup 3, forward fit 1, adjoint 1, inward fit 1
LAUNCHES_PER_STEP = 5 + 2 + 3 + 1 + 1 + 1


def path_summary(r, workload, dev, max_mhz=None):
    """Throughput, stage times, end-to-end figure and the building kernel's
    FP32 roofline of one time_path result."""
    steps, total_ms = r["steps"], r["total_ms"]
    st = r["stats"]
    b_ms = r["stage"]["build"]
    alg_flops = (st["nav_tests"] * FLOPS_NAV_TEST + st["cand_steps"] * FLOPS_CAND_STEP
                 + st["chi2_evals"] * FLOPS_BOX + st["chi2_full"] * FLOPS_CHI2 + st["updates"] * FLOPS_UPDATE)
    achieved = alg_flops / (b_ms * 1e-3) / 1e12
    peak = fp32_peak(dev, max_mhz)
    return {
        "value": r["units"] * steps / (total_ms * 1e-3), "unit": UNIT, "ms_per_step": total_ms / steps,
        "config": {"workload": WORKLOADS[workload], "events_per_step_per_gpu": r["n_events"], "tracks": r["S"],
                   "hits": r["n_hits"], "surfaces": r["L"], "max_cands": r["max_cands"],
                   "l2": "flushed (256 MB write) between timed steps", "adjoint_in_step": True,
                   "launch": "cuda_graph" if r["use_graph"] else "eager", "tuned": r["tuned"]},
        "events_per_s": r["n_events"] * steps / (total_ms * 1e-3),
        "fit_tracks_per_s": r["S"] * steps / (total_ms * 1e-3),
        "stage_ms": r["stage"],
        "roofline": {"kernel": "k_build (combinatorial building)", "bound": "alu", "achieved": achieved,
                     "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": profiled_traffic("k_build_%s" % workload),
                     "peak_basis": FP32_PEAK_BASIS, "algorithmic_flops_per_launch": alg_flops,
                     "build_ms": b_ms},
        "e2e": {"value": r["units"] * steps / (r["e2e_total_ms"] * 1e-3), "unit": UNIT,
                "h2d_bytes_per_step": r["h2d"], "d2h_bytes_per_step": r["d2h"],
                "ms_per_step": r["e2e_total_ms"] / steps},
        "gpu_launches": LAUNCHES_PER_STEP * steps,
        "launch_ms_per_step": {"eager": r["eager_ms"] / steps,
                               "cuda_graph": None if r["graph_ms"] is None else r["graph_ms"] / steps,
                               "graph_note": r["graph_note"]},
        "work": st,
        "binning_roofline": binning_roofline(r),
    }


def binning_roofline(r):
    """HBM roofline of the binning stage (its five kernels) of one step."""
    tu = r.get("tuned") or {}
    n_bins = int(r["n_events"]) * int(r["L"]) * int(tu.get("n_phi", 64)) * int(tu.get("n_w", 16))
    ms = r["stage"]["bin"]
    byts = r["n_hits"] * BYTES_BIN_HIT + n_bins * BYTES_BIN_BIN
    hbm = measured_peaks().get("hbm_gbs", 6800.0)
    gbs = byts / (ms * 1e-3) / 1e9 if ms > 0 else None
    return {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": None if gbs is None else gbs / hbm,
            "algorithmic_bytes": byts, "bins": n_bins, "ms": ms,
            "note": "bins = events x layers x tuned phi x w bins (every layer binned alike)"}


def c1_latency(r):
    """C1 is launch-latency bound: the whole path on its one 100-track event in
    microseconds per event."""
    steps = r["steps"]
    return {"workload": WORKLOADS["c1"], "us_per_event": 1e3 * r["total_ms"] / steps,
            "us_per_event_eager": 1e3 * r["eager_ms"] / steps,
            "us_per_event_cuda_graph": None if r["graph_ms"] is None else 1e3 * r["graph_ms"] / steps,
            "us_per_event_e2e": 1e3 * r["e2e_total_ms"] / steps,
            "launch": "cuda_graph" if r["use_graph"] else "eager", "cand_steps": r["stats"]["cand_steps"],
            "stage_us": {k: 1e3 * v for k, v in r["stage"].items()}}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import numpy as np
    import torch

    import synth
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if args.only:
        import paper_2002_06295_gb300 as mkf_only
        dev_only = torch.device("cuda", local)
        fn = {"strips": measure_strips, "seeding": measure_seeding, "overlaps": measure_overlaps,
              "in_flight": measure_in_flight, "fit_gradient": measure_fit_gradient}[args.only]
        print(json.dumps({args.only: fn(mkf_only, dev_only)}), flush=True)
        return
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if dist:
        dist.barrier()
    import paper_2002_06295_gb300 as mkf

    # CPU baseline first (spawned workers, before any heavy GPU work)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = n_cores()
        pool = oracle_pool(cores)
        per = args.cpu_sample_seeds or 5000
        u, dt = oracle_step(pool, cores, per, 0)
        pool.close()
        pool1 = oracle_pool(1)   # the same oracle on one core, on a smaller sample
        per1 = max(1, per // 16)
        u1, dt1 = oracle_step(pool1, 1, per1, 0)
        pool1.close()
        cpu = {"value": u / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "%d of the 5000 seeds of the C2 event (building only, FP64, brute-force hit search), "
                         "one process per core, %.1f s wall" % (per, dt),
               "one_core": {"value": u1 / dt1, "unit": UNIT, "cores": 1,
                            "sample": "%d seeds of the same event, %.1f s" % (per1, dt1)}}

    dev = torch.device("cuda", local)
    cfg_id = {"c2": 2, "c3": 3, "c5": 5}[args.workload]
    evs = workload_events(synth, cfg_id, rank, world)
    clocks = ClockSampler(local)
    r = time_path(mkf, dev, evs, synth.WORKLOAD_SPECS[cfg_id], args.steps, args.warmup, dist=dist, clocks=clocks,
                  graph=not args.no_graph)
    clk = r["clocks"]
    if rank != 0:
        return
    secondary = None
    if world == 1 and not args.no_secondary:
        from paper_2002_06295_gb300 import tune as _tune
        secondary = {}
        if args.workload != "c5":
            secondary["stress_c5"] = path_summary(
                time_path(mkf, dev, workload_events(synth, 5, 0), synth.WORKLOAD_SPECS[5], min(args.steps, 5), 3),
                "c5", dev)
        if args.workload == "c2":
            secondary["c2_in_flight"] = measure_in_flight(mkf, dev)
        secondary["c1_event"] = c1_latency(
            time_path(mkf, dev, workload_events(synth, 1, 0), synth.WORKLOAD_SPECS[1], 50, 5))
        secondary.update({"batched_vs_plain": measure_batched(mkf, _tune, dev),
                          "fit_gradient": measure_fit_gradient(mkf, dev),
                          "strip_clustering": measure_strips(mkf, dev),
                          "seeding": measure_seeding(mkf, dev),
                          "overlaps": measure_overlaps(mkf, dev)})
    summ = path_summary(r, args.workload, dev, clk.get("sm_max_mhz"))
    line = {
        "metric": METRIC, "value": summ["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": summ["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": summ["config"],
        "events_per_s": world * summ["events_per_s"],
        "fit_tracks_per_s": world * summ["fit_tracks_per_s"],
        "stage_ms": summ["stage_ms"],
        "work": r["stats"],
        "roofline": summ["roofline"],
        "binning_roofline": summ["binning_roofline"],
        "cpu_baseline": cpu,
        "e2e": summ["e2e"],
        "gpu_launches": summ["gpu_launches"],
        "launch_ms_per_step": summ["launch_ms_per_step"],
        "secondary": secondary,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
