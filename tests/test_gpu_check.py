"""The debug library (FKD_CHECK=1) on a GPU: the small parity cases of
tests/check_cases.py -- streams in every mask mode, keypoint binning in
spans, scale-space suppression, per-pixel masks, ragged and tiny frames,
description and a group tick mix -- run with every kernel checking its
memory indices (a failure would be an FkdError naming the access) and the
allocations' guard bands checked after each case, and still equal the
oracle. A process of its own: the binding loads one library per process."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_debug_build_checks_indices_and_guard_bands():
    env = dict(os.environ, FKD_CHECK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "check_cases.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "check cases ok" in r.stdout
