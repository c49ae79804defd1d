"""The debug build's bounds checks on the GPU: every part of the hot path run
through libfewha_debug.so (FEWHA_DEBUG=1, in a child process so that this
process keeps the release library) records no out-of-bounds index and
matches the FP64 oracle within each path's tolerance."""

import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def test_debug_build_records_no_violation_and_matches_oracle():
    lib = os.path.join(os.path.dirname(HERE), "paper_2009_00946_b300", "libfewha_debug.so")
    assert os.path.exists(lib), "the debug library is built next to the release library"
    env = dict(os.environ, FEWHA_DEBUG="1")
    p = subprocess.run([sys.executable, os.path.join(HERE, "debug_bounds_run.py")], env=env, capture_output=True,
                       text=True, timeout=900)
    assert p.returncode == 0, p.stderr[-3000:]
    res = json.loads(p.stdout.strip().splitlines()[-1])
    assert res["debug_build"], "FEWHA_DEBUG=1 must load the debug build"
    assert len(res["cases"]) >= 15
    for name, rec in res["cases"].items():
        assert rec.get("exception") is None, (name, rec)
        assert rec["count"] == 0, (name, rec)
        assert rec["err"] is not None and rec["err"] < rec["tol"], (name, rec)
