"""The multi-rank path of bench.py on CPU: two gloo ranks on 127.0.0.1.

The bench runs one replica of the workload per rank (no collective on the data
path); its only cross-rank steps are the barriers around the timed region and
the reductions that turn per-rank units and times into the whole-job rate
(units of all ranks over the slowest rank's time).  The reference arm runs on
rank 0 alone.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys
sys.path.insert(0, sys.argv[1])
import bench
rank, world, _ = bench.dist_setup(False)
bench.barrier(world)
out = {
    "rank": rank,
    "max": bench.max_over_ranks(float(rank + 1), world),
    "sum": bench.reduce_over_ranks(float(rank + 1), world, "sum"),
    "rate": bench.job_rate(10.0 * (rank + 1), float(rank + 1), world),
}
bench.barrier(world)
print(json.dumps(out), flush=True)
"""


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _launch(argv, world=2, timeout=300):
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen(argv, env=env, cwd=ROOT, stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                      text=True))
    outs = []
    for p in procs:
        try:
            o, e = p.communicate(timeout=timeout)
        except subprocess.TimeoutExpired:
            p.kill()
            o, e = p.communicate()
        outs.append((p.returncode, o, e))
    return outs


def test_rank_reductions_give_the_whole_job_rate():
    outs = _launch([sys.executable, "-c", WORKER, ROOT])
    for rc, o, e in outs:
        assert rc == 0, e[-2000:]
    res = sorted((json.loads(o.strip().splitlines()[-1]) for _, o, _ in outs), key=lambda d: d["rank"])
    for d in res:
        assert d["max"] == 2.0
        assert d["sum"] == 3.0
        assert d["rate"] == pytest.approx(30.0 / 2.0)      # 10 + 20 units over the slower rank's 2 s


def test_reference_arm_runs_on_rank_zero_only():
    outs = _launch([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                    "--warmup", "0"])
    for rc, o, e in outs:
        assert rc == 0, e[-2000:]
    lines0 = [l for l in outs[0][1].splitlines() if l.startswith("{")]
    lines1 = [l for l in outs[1][1].splitlines() if l.startswith("{")]
    assert len(lines0) == 1 and not lines1
    d = json.loads(lines0[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
