"""The bounds-checked build (libbttb_checked.so, -DBTTB_CHECKED=1), the stand-in for a memory checker.

Its kernels check the global accesses of the vector loads and stores, the bulk and asynchronous copies,
the Arnoldi / Givens / GEMM-epilogue accesses and the cluster exchanges against the device buffers the
library allocated or was handed; a failed check is counted and the access skipped, so nothing faults.
The workload (tests/checked_workload.py) runs in a child process that loads the checked library: every
product form and precision, the many-column GEMMs, the solver variants, block-Jacobi and the
allocation-free product, each against the oracle.  A positive control first reads one element past a
buffer of the library's own through a checked load and sees exactly one counted (and skipped) access.
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_finds_nothing_out_of_bounds():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_20350_gb300 import build
    build.build(checked=True)
    env = dict(os.environ, BTTB_LIB_CHECKED="1", PYTHONPATH=ROOT + os.pathsep + os.path.join(ROOT, "tests"))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checked_workload.py")], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["probe_hits"] == 1, out            # the checks see an out-of-bounds read (and skip it)
    assert out["hits"] == 0, f"out-of-bounds accesses: {out['hits']}, first at {out['first']:#x}; {out['bad']}"
    assert not out["bad"], out["bad"]             # and every result still matches the oracle
    assert out["cases"] >= 60
