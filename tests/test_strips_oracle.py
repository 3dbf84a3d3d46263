"""Pins of the strip-clustering oracle (Sec. 4): hand-built modules for each
rule, and an independent formulation (run segmentation of the strip classes)
on random modules."""
import itertools

import numpy as np
import pytest

import synth.strips as strips


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def _one(orc, adc, noise=5.0, bad=(), max_bad_gap=1, q_min=30):
    a = np.array([adc], np.uint16)
    nq = np.full_like(a, int(round(8 * noise)))
    b = np.zeros_like(a, dtype=np.uint8)
    for i in bad:
        b[0, i] = 1
    r = orc.strip_clusters(a, nq, b, max_bad_gap=max_bad_gap, q_min=q_min)
    return [(int(f), int(l), int(c)) for f, l, c in zip(r["first"], r["last"], r["charge"])], r


def test_single_seed_strip(orc):
    cl, r = _one(orc, [0, 0, 40, 0, 0])            # 8 sigma: seed; 40 > 25 sigma^2 quadrature test passes
    assert cl == [(2, 2, 40)] and r["center"][0] == 2.0


def test_no_seed_no_cluster(orc):
    cl, _ = _one(orc, [0, 14, 14, 14, 0])          # 2.8 sigma strips: candidates, but no 3-sigma seed
    assert cl == []


def test_quadrature_rule(orc):
    # one 3.2-sigma seed with 2.5-sigma neighbours: sum a^2 = (16^2 + 2*12.5^2) < 25 * 3 * 25
    cl, _ = _one(orc, [0, 12, 16, 12, 0], q_min=0)
    assert cl == []
    # a strong seed passes: 64 * (50^2 + 2 * 12^2) > 25 * 3 * 40^2
    cl, _ = _one(orc, [0, 12, 50, 12, 0])
    assert cl == [(1, 3, 74)]


def test_minimum_charge(orc):
    cl, _ = _one(orc, [0, 0, 40, 0, 0], q_min=41)
    assert cl == []


def test_gap_rules(orc):
    sig = [0, 30, 0, 30, 0]
    assert _one(orc, sig)[0] == [(1, 1, 30), (3, 3, 30)]                     # good strip below threshold splits
    assert _one(orc, sig, bad=[2])[0] == [(1, 3, 60)]                        # one bad strip is bridged
    sig2 = [0, 30, 0, 0, 30, 0]
    assert _one(orc, sig2, bad=[2, 3])[0] == [(1, 1, 30), (4, 4, 30)]        # two bad strips are not (gap 1)
    assert _one(orc, sig2, bad=[2, 3], max_bad_gap=2)[0] == [(1, 4, 60)]
    # a bad strip above threshold adds nothing; bad strips at the edges are not part of a cluster
    assert _one(orc, [0, 30, 900, 30, 0], bad=[2])[0] == [(1, 3, 60)]
    assert _one(orc, [30, 0, 0], bad=[1])[0] == [(0, 0, 30)]


def test_module_edges(orc):
    cl, r = _one(orc, [40, 20, 0, 0, 20, 40])
    assert cl == [(0, 1, 60), (4, 5, 60)]
    assert abs(r["center"][0] - 20.0 / 60.0) < 1e-15 and abs(r["center"][1] - (80.0 + 200.0) / 60.0) < 1e-15


def _segment_reference(adc, nq, bad, max_bad_gap, q_min):
    """Independent formulation: classify each strip (C candidate, B bad, N
    neither), split the module at N and at runs of B longer than the allowed
    gap, drop the B at both ends of a piece; a piece with a C is a cluster
    candidate, judged by the seed, quadrature and charge rules."""
    out = []
    M, N = adc.shape
    for m in range(M):
        cls = ["B" if bad[m, i] else ("C" if 8 * int(adc[m, i]) > 2 * int(nq[m, i]) else "N") for i in range(N)]
        pieces, cur, i = [], [], 0
        for key, grp in itertools.groupby(range(N), key=lambda j: cls[j]):
            idx = list(grp)
            if key == "N" or (key == "B" and len(idx) > max_bad_gap):
                if cur:
                    pieces.append(cur)
                cur = []
            else:
                cur.extend(idx)
        if cur:
            pieces.append(cur)
        for p in pieces:
            c = [j for j in p if cls[j] == "C"]
            if not c:
                continue
            a = np.array([int(adc[m, j]) for j in c], np.int64)
            n = np.array([int(nq[m, j]) for j in c], np.int64)
            if not (8 * a > 3 * n).any() or not 64 * (a * a).sum() > 25 * (n * n).sum() or a.sum() < q_min:
                continue
            out.append((m, c[0], c[-1], int(a.sum()), float((np.array(c) * a).sum() / a.sum())))
    return out


@pytest.mark.parametrize("gap", [0, 1, 2])
def test_oracle_equals_segmentation_on_random_modules(orc, gap):
    rng = np.random.default_rng(30 + gap)
    nq, bad = strips.make_strip_calibration(60, 256, rng, bad_frac=0.05)
    adc = strips.make_strip_event(nq, rng, occupancy=0.04)
    ref = _segment_reference(adc, nq, bad, gap, 30)
    r = orc.strip_clusters(adc, nq, bad, max_bad_gap=gap, q_min=30)
    got = list(zip(r["module"].tolist(), r["first"].tolist(), r["last"].tolist(), r["charge"].tolist(),
                   r["center"].tolist()))
    assert len(ref) > 50
    assert [g[:4] for g in got] == [x[:4] for x in ref]
    assert np.allclose([g[4] for g in got], [x[4] for x in ref], rtol=0, atol=1e-12)
