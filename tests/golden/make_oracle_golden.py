"""Writes oracle_c1.json: the FP64 oracle's results on the seeded C1 event
(combinatorial building with duplicate removal, then the outward and inward
fit of the kept tracks).  The paper prints no worked example with inputs and
outputs, so the stored values are the oracle's own: a regression fixture that
makes any change to the oracle's arithmetic show up as a changed stored value.
Calls only oracle/ and synth/ (the seeded input generator).

    python tests/golden/make_oracle_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402

SPEC = dict(chi2_cut=30.0, max_cands=4, max_holes=3, min_hits=4, dup_frac=0.5)


def compute():
    ev = synth.make_config_event(1)
    geo = oracle.Geo.of(ev.geom)
    b = oracle.build_event(geo, ev.hit_xyz, ev.hit_lcov, ev.hit_layer, ev.seed_par, ev.seed_cov, **SPEC)
    kept = np.nonzero(b["flags"] == 1)[0]
    hits = b["hits"][kept]
    fpar, fcov, fchi2, fok = oracle.fit(geo, ev.hit_xyz, ev.hit_lcov, ev.hit_layer, hits, ev.seed_par[kept],
                                        ev.seed_cov[kept])
    bpar, bcov, bchi2, bok = oracle.fit(geo, ev.hit_xyz, ev.hit_lcov, ev.hit_layer, hits, fpar, fcov, direction=-1)
    return {
        "event": "C1 (synth.make_config_event(1)), oracle.build_event with %s" % json.dumps(SPEC),
        "build": {k: b[k].tolist() for k in ("hits", "nhits", "nholes", "flags", "fragile", "chi2", "par")},
        "build_stats": b["stats"],
        "kept": kept.tolist(),
        "fit_outward": {"par": fpar.tolist(), "chi2": fchi2.tolist(), "ok": fok.tolist()},
        "fit_inward": {"par": bpar.tolist(), "chi2": bchi2.tolist(), "ok": bok.tolist()},
    }


if __name__ == "__main__":
    with open(os.path.join(HERE, "oracle_c1.json"), "w") as f:
        json.dump(compute(), f, sort_keys=True, separators=(",", ":"))
        f.write("\n")
