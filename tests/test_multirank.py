"""The multi-rank logic of bench.py on CPU: two gloo ranks (127.0.0.1), each
with its own numbers, must agree on the slowest rank's times, the sum of the
work of all ranks and a launch decision taken only if every rank can."""
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
