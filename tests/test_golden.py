"""The oracle against its stored results on the seeded C1 event
(tests/golden/oracle_c1.json, written by tests/golden/make_oracle_golden.py):
discrete results exactly on the seeds whose decisions have a margin (the
oracle marks the others fragile), continuous results to 1e-9 relative, which
allows for FMA contraction on another host but not for a changed formula."""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))


def test_oracle_matches_stored_c1_results():
    import make_oracle_golden as mg
    with open(os.path.join(HERE, "golden", "oracle_c1.json")) as f:
        ref = json.load(f)
    now = json.loads(json.dumps(mg.compute()))
    assert now["event"] == ref["event"]
    rb, nb = ref["build"], now["build"]
    firm = ~np.array(rb["fragile"], bool)
    assert firm.mean() > 0.9
    for k in ("hits", "nhits", "nholes", "flags"):
        assert np.array_equal(np.array(nb[k])[firm], np.array(rb[k])[firm]), k
    for k in ("chi2", "par"):
        assert np.allclose(np.array(nb[k])[firm], np.array(rb[k])[firm], rtol=1e-9, atol=1e-12), k
    # kept tracks and their fits, compared per seed over the firm seeds
    kr, kn = np.array(ref["kept"]), np.array(now["kept"])
    assert set(kr[firm[kr]].tolist()) == set(kn[firm[kn]].tolist())
    rows_r = {int(sd): i for i, sd in enumerate(kr)}
    rows_n = {int(sd): i for i, sd in enumerate(kn)}
    common = [sd for sd in rows_r if firm[sd] and sd in rows_n]
    assert len(common) > 0.9 * len(kr)
    ir = [rows_r[sd] for sd in common]
    inn = [rows_n[sd] for sd in common]
    for fit in ("fit_outward", "fit_inward"):
        assert np.array_equal(np.array(now[fit]["ok"])[inn], np.array(ref[fit]["ok"])[ir]), fit
        for k in ("par", "chi2"):
            assert np.allclose(np.array(now[fit][k])[inn], np.array(ref[fit][k])[ir], rtol=1e-9, atol=1e-12), (fit, k)
