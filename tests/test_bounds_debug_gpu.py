"""The bounds-checking debug build (a compute-sanitizer stand-in): built with
KS_DEBUG_BOUNDS, its FP32 kernels and the split-K reduction check every global
access against the operands' extents.  tests/bounds_debug_check.py drives it in
a child process (the binding selects the debug build by environment)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_no_access_outside_the_operands():
    from paper_2008_13145_gb300 import build
    build.build_debug_library()
    env = {**os.environ, "KSELECT_DEBUG_BOUNDS": "1"}
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "bounds_debug_check.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert res["configs"] >= 90 and res["split_configs"] >= 20, res
    assert res["out_of_bounds"] == 0, res
    assert res["worst_error_ratio"] <= 1e-5, res
    assert res["negative_control_flagged"] > 0, res
