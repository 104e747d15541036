"""Multi-rank host logic of bench.py on the CPU: two gloo ranks agree on the
slowest rank's time per step, and the whole-job rate counts every rank's
flops over that time (independent replicas, weak scaling)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RANK_SCRIPT = """
import json, sys
sys.path.insert(0, {root!r})
import torch.distributed as dist
dist.init_process_group("gloo")
import bench
r, w = dist.get_rank(), dist.get_world_size()
ms = bench.slowest_rank_ms(10.0 + 5.0 * r, dist, "cpu")
print(json.dumps({{"rank": r, "ms": ms, "gflops": bench.job_gflops(3e9, w, ms)}}), flush=True)
dist.barrier()
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_take_the_slowest_rank():
    port = _free_port()
    script = RANK_SCRIPT.format(root=ROOT)
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", script], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    try:
        for p in procs:
            out, err = p.communicate(timeout=120)
            assert p.returncode == 0, err[-2000:]
            outs.append(json.loads(out.strip().splitlines()[-1]))
    finally:
        for p in procs:
            if p.poll() is None:
                p.kill()
    assert sorted(o["rank"] for o in outs) == [0, 1]
    for o in outs:
        assert o["ms"] == 15.0                                     # rank 1 is the slower one
        assert o["gflops"] == pytest.approx(2 * 3e9 / 15e-3 / 1e9)  # both ranks' flops


def test_one_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.slowest_rank_ms(12.5, None, "cpu") == 12.5
    assert bench.job_gflops(2e9, 1, 10.0) == pytest.approx(200.0)
