"""Strip clustering on the GPU (Sec. 4) against the oracle: every cluster
(row, first and last strip, charge exactly; the charge-weighted centre within
1e-6) for every work split of the TMA kernel, widths that are a multiple of
the chunk, of 16 only (ragged last chunk), and of neither (plain kernel), an
unaligned ADC base (plain kernel), allowed gaps 0..2, event counts that do not
fill the last work item, the full 16-event workload the benchmark times, and
the capacity report."""
import numpy as np
import pytest
import torch

import synth.strips as strips

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _oracle(evs, nq, bad, gap, q_min):
    import oracle
    M = nq.shape[0]
    ref = []
    for e, a in enumerate(evs):
        r = oracle.strip_clusters(a, nq, bad, max_bad_gap=gap, q_min=q_min)
        r["row"] = r["module"] + e * M
        ref.append(r)
    return {k: np.concatenate([r[k] for r in ref]) for k in ("row", "first", "last", "charge", "center")}


def _compare(o, n, ref):
    assert n == ref["row"].size
    got = {k: o[k][:n].cpu().numpy() for k in ("row", "first", "last", "charge", "center")}
    order = np.lexsort((got["first"], got["row"]))
    for k in ("row", "first", "last", "charge"):
        assert np.array_equal(got[k][order], ref[k]), k
    assert np.allclose(got["center"][order], ref["center"], rtol=1e-6, atol=0)


def _run(n_modules, n_strips, n_events, gap, seed, config=(0, 0, 0), max_out=None, offset=0):
    import paper_2002_06295_gb300 as mkf
    rng = np.random.default_rng(seed)
    nq, bad = strips.make_strip_calibration(n_modules, n_strips, rng, bad_frac=0.03)
    evs = [strips.make_strip_event(nq, rng, occupancy=0.02) for _ in range(n_events)]
    dev = torch.device("cuda", 0)
    ctx = mkf.Context(0)
    mkf.mkf_set_strip_config(ctx, *config)
    flat = np.concatenate(evs, 0).reshape(-1)
    buf = torch.zeros(flat.size + offset, dtype=torch.uint16, device=dev)
    buf[offset:] = torch.from_numpy(flat).to(dev)
    adc = buf[offset:].view(n_events * n_modules, n_strips)
    o = mkf.mkf_cluster_strips(ctx, adc, torch.from_numpy(nq).to(dev), torch.from_numpy(bad).to(dev),
                               max_bad_gap=gap, q_min=30, max_out=max_out)
    n = int(o["count"].item())
    return ctx, o, n, _oracle(evs, nq, bad, gap, 30)


_SPLITS = ((32, 1, 1), (32, 1, 2), (32, 1, 3), (32, 1, 4), (32, 2, 2), (64, 1, 2), (64, 1, 3), (64, 2, 2))


@pytest.mark.parametrize("n_strips,gap,config", [(768, 1, c) for c in _SPLITS] + [
    (720, 2, (32, 2, 2)), (720, 0, (64, 2, 2)), (720, 1, (32, 1, 3)), (512, 2, (0, 0, 0)), (500, 1, (0, 0, 0)),
])
def test_clusters_equal_oracle(n_strips, gap, config):
    import paper_2002_06295_gb300 as mkf
    ctx, o, n, ref = _run(3000, n_strips, 3, gap, seed=40 + gap + n_strips, config=config)
    assert n > 10000
    mkf.mkf_sync(ctx)
    _compare(o, n, ref)
    ctx.close()


def test_unaligned_base_takes_plain_kernel():
    import paper_2002_06295_gb300 as mkf
    ctx, o, n, ref = _run(1000, 768, 2, 1, seed=48, offset=1)
    mkf.mkf_sync(ctx)
    _compare(o, n, ref)
    ctx.close()


def test_full_workload_equals_oracle():
    """The 16-event, 15000-module, 768-strip batch of the benchmark (4 distinct
    events, each used 4 times), default work split."""
    import paper_2002_06295_gb300 as mkf
    rng = np.random.default_rng(20026)
    M, N, E = 15000, 768, 16
    nq, bad = strips.make_strip_calibration(M, N, rng)
    base = [strips.make_strip_event(nq, rng) for _ in range(4)]
    evs = [base[e % 4] for e in range(E)]
    dev = torch.device("cuda", 0)
    ctx = mkf.Context(0)
    o = mkf.mkf_cluster_strips(ctx, torch.from_numpy(np.concatenate(evs, 0)).to(dev), torch.from_numpy(nq).to(dev),
                               torch.from_numpy(bad).to(dev), max_out=4 << 20)
    n = int(o["count"].item())
    mkf.mkf_sync(ctx)
    _compare(o, n, _oracle(evs, nq, bad, 1, 30))
    ctx.close()


def test_capacity_is_reported():
    import paper_2002_06295_gb300 as mkf
    ctx, o, n, ref = _run(200, 768, 1, 1, seed=47, max_out=10)
    assert n == ref["row"].size > 10
    with pytest.raises(mkf.MkfError):
        mkf.mkf_sync(ctx)
    ctx.close()


def test_splits_match_binding():
    import paper_2002_06295_gb300.api as api
    assert tuple(api.STRIP_SPLITS) == _SPLITS


def test_bad_config_rejected():
    import paper_2002_06295_gb300 as mkf
    ctx = mkf.Context(0)
    with pytest.raises(mkf.MkfError):
        mkf.mkf_set_strip_config(ctx, 64, 4, 2)
    ctx.close()


@pytest.mark.parametrize("n_strips,gap,bad_frac,config", [
    (16, 1, 0.03, (32, 1, 2)),      # one ragged chunk
    (768, 40, 0.5, (32, 1, 2)),     # half the strips bad, gaps longer than a 32-strip block
    (768, 40, 0.5, (64, 2, 2)),
    (512, 0, 0.5, (0, 0, 0)),
])
def test_extreme_gaps_and_widths(n_strips, gap, bad_frac, config):
    import oracle
    import paper_2002_06295_gb300 as mkf
    rng = np.random.default_rng(90 + gap + n_strips)
    nq, bad = strips.make_strip_calibration(400, n_strips, rng, bad_frac=bad_frac)
    evs = [strips.make_strip_event(nq, rng, occupancy=0.05) for _ in range(2)]
    dev = torch.device("cuda", 0)
    ctx = mkf.Context(0)
    mkf.mkf_set_strip_config(ctx, *config)
    o = mkf.mkf_cluster_strips(ctx, torch.from_numpy(np.concatenate(evs, 0)).to(dev), torch.from_numpy(nq).to(dev),
                               torch.from_numpy(bad).to(dev), max_bad_gap=gap, q_min=30)
    n = int(o["count"].item())
    mkf.mkf_sync(ctx)
    _compare(o, n, _oracle(evs, nq, bad, gap, 30))
    ctx.close()


def test_default_split_for_many_events():
    """From 32 events up the default takes two events per item."""
    import paper_2002_06295_gb300 as mkf
    ctx, o, n, ref = _run(200, 768, 40, 1, seed=77)
    mkf.mkf_sync(ctx)
    _compare(o, n, ref)
    ctx.close()


def test_no_events():
    import paper_2002_06295_gb300 as mkf
    dev = torch.device("cuda", 0)
    ctx = mkf.Context(0)
    nq = torch.full((10, 768), 32, dtype=torch.uint16, device=dev)
    bad = torch.zeros((10, 768), dtype=torch.uint8, device=dev)
    o = mkf.mkf_cluster_strips(ctx, torch.zeros((0, 768), dtype=torch.uint16, device=dev), nq, bad, max_out=16)
    assert int(o["count"].item()) == 0
    mkf.mkf_sync(ctx)
    ctx.close()
