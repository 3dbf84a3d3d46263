"""The multi-rank logic of bench.py on CPU: two gloo ranks (127.0.0.1), each
with its own numbers, must agree on the slowest rank's times, the sum of the
work of all ranks and a launch decision taken only if every rank can; and the
event sharding itself: each rank builds its contiguous range of a batch (the
oracle stands in for the GPU here), the results gathered on rank 0 equal one
single-rank run over the whole batch."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RANK_SCRIPT = r'''
import os, sys, json
sys.path.insert(0, sys.argv[1])
import torch, torch.distributed as dist
import bench
dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%s" % sys.argv[2],
                        rank=int(sys.argv[3]), world_size=2)
r = dist.get_rank()
dev = torch.device("cpu")
times = bench.rank_reduce(dist, dev, [1.5 + r, 7.0 - 3 * r], "max")
work = bench.rank_reduce(dist, dev, [1000 + 234 * r], "sum")
ok = bench.rank_reduce(dist, dev, [1 if r == 0 else 0], "min")
alone = bench.rank_reduce(None, dev, [3.0], "sum")
print(json.dumps(dict(rank=r, times=times, work=work, ok=ok, alone=alone)))
dist.destroy_process_group()
'''


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_rank_reduce_two_gloo_ranks():
    import json
    port = str(_free_port())
    procs = [subprocess.Popen([sys.executable, "-c", RANK_SCRIPT, ROOT, port, str(r)], stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True) for r in range(2)]
    outs = []
    for p in procs:
        try:
            o, e = p.communicate(timeout=120)
        except subprocess.TimeoutExpired:
            for q in procs:
                q.kill()
            pytest.fail("gloo ranks did not finish")
        assert p.returncode == 0, e
        outs.append(json.loads(o.strip().splitlines()[-1]))
    for o in outs:
        assert o["times"] == [2.5, 7.0]       # slowest rank per entry
        assert o["work"] == [2234.0]          # all ranks' work
        assert o["ok"] == [0.0]               # rank 1 cannot: nobody does
        assert o["alone"] == [3.0]            # one rank: identity


SHARD_SCRIPT = r'''
import os, sys, json
sys.path.insert(0, sys.argv[1])
import numpy as np
import torch.distributed as dist
import bench, oracle, synth
dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%s" % sys.argv[2],
                        rank=int(sys.argv[3]), world_size=2)
r = dist.get_rank()
N = 5                                     # a batch of five C1-geometry events
start, end = bench.shard_range(N, r, 2)
local = []
for e in range(start, end):
    ev = synth.make_config_event(1, e)
    o = oracle.build_event(oracle.Geo.of(ev.geom), ev.hit_xyz, ev.hit_lcov, ev.hit_layer, ev.seed_par,
                           ev.seed_cov, max_cands=4)
    local.append(dict(event=e, hits=o["hits"].tolist(), flags=o["flags"].tolist(), par=o["par"].tolist()))
got = bench.gather_results(dist, dict(rank=r, range=[start, end], events=local))
if r == 0:
    print(json.dumps(got))
dist.destroy_process_group()
'''


def test_event_sharding_two_gloo_ranks_equals_one_rank():
    import json
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    import synth
    # the ranges of any split are contiguous, disjoint and cover every event
    for n, w in ((5, 2), (256, 8), (3, 4), (0, 2)):
        rs = [bench.shard_range(n, r, w) for r in range(w)]
        assert rs[0][0] == 0 and rs[-1][1] == n
        assert all(rs[i][1] == rs[i + 1][0] for i in range(w - 1))
        assert max(b - a for a, b in rs) - min(b - a for a, b in rs) <= 1
    port = str(_free_port())
    procs = [subprocess.Popen([sys.executable, "-c", SHARD_SCRIPT, ROOT, port, str(r)], stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True) for r in range(2)]
    outs = []
    for p in procs:
        try:
            o, e = p.communicate(timeout=300)
        except subprocess.TimeoutExpired:
            for q in procs:
                q.kill()
            pytest.fail("gloo ranks did not finish")
        assert p.returncode == 0, e
        outs.append(o)
    gathered = json.loads(outs[0].strip().splitlines()[-1])
    assert [g["rank"] for g in gathered] == [0, 1]
    assert [g["range"] for g in gathered] == [[0, 3], [3, 5]]
    merged = [ev for g in gathered for ev in g["events"]]
    assert [ev["event"] for ev in merged] == list(range(5))
    for ev_out in merged:
        ev = synth.make_config_event(1, ev_out["event"])
        ref = oracle.build_event(oracle.Geo.of(ev.geom), ev.hit_xyz, ev.hit_lcov, ev.hit_layer, ev.seed_par,
                                 ev.seed_cov, max_cands=4)
        assert np.array_equal(np.array(ev_out["hits"]), ref["hits"])
        assert np.array_equal(np.array(ev_out["flags"]), ref["flags"])
        assert np.array_equal(np.array(ev_out["par"]), ref["par"])
