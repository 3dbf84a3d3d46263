"""The synthetic workloads keep the shapes their descriptions give (CPU):
layer counts, tracks per event, the noise fraction read as a fraction of the
signal hits, and the resulting hit counts; the generator is deterministic for
a given (configuration, event)."""
import numpy as np

import synth


def _signal(ev):
    return int((ev.true_hits >= 0).sum())


def test_plain_events_sizes():
    e1 = synth.make_config_event(1)
    assert e1.geom.n_layers == 10 and e1.n_seeds == 100 and e1.n_hits == _signal(e1)
    e2 = synth.make_config_event(2)
    assert e2.geom.n_layers == 38 and e2.n_seeds == 5000
    sig = _signal(e2)
    assert e2.n_hits - sig == round(0.2 * sig)          # 20 % noise, of the signal hits
    assert 80_000 < e2.n_hits < 90_000                  # "order of 100k hits"
    assert 12.0 < sig / e2.n_seeds < 16.0


def test_stress_event_sizes():
    e5 = synth.make_config_event(5)
    assert e5.geom.n_layers == 10 and e5.n_seeds == 10000
    sig = _signal(e5)
    assert e5.n_hits - sig == round(0.5 * sig)          # 50 % noise, of the signal hits
    assert 85_000 < e5.n_hits < 100_000


def test_batched_multiplicities():
    n = np.array([synth.make_config_event(3, k).n_seeds for k in range(24)])
    assert n.min() >= 200 and n.max() <= 8000 and len(set(n.tolist())) > 20   # uneven, log-uniform 200..8000


def test_generator_is_deterministic():
    a, b = synth.make_config_event(2), synth.make_config_event(2)
    assert np.array_equal(a.hit_xyz, b.hit_xyz) and np.array_equal(a.hit_layer, b.hit_layer)
    assert np.array_equal(a.seed_par, b.seed_par) and np.array_equal(a.true_hits, b.true_hits)
    c = synth.make_config_event(2, 1)
    assert not np.array_equal(a.hit_xyz[:100], c.hit_xyz[:100])
