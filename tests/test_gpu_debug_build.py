"""The bounds-checked debug build (compiled with -DPMF_DEBUG; it stands in
for compute-sanitizer, which this pool does not offer): the small workload's
whole forward + adjoint and the Stage-1 rasterizer run through it in a fresh
process with guard bands around every caller buffer; no bounds check may fail,
no guard byte may change, and the results must match the oracle."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_debug_build_runs_the_step_with_no_failed_check_and_intact_guards():
    env = dict(os.environ, PMF_LIB_VARIANT="debug")
    r = subprocess.run([sys.executable, "-m", "tests.debug_step"], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=1200)
    print(r.stdout[-2000:])
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-4000:]
    assert "DEBUG-STEP-OK" in r.stdout
