"""The debug build's device-side range checks stay silent on valid work.

A child process loads libhx_debug.so (HX_DEBUG=1), runs every entry point on
ragged, misaligned, multi-round and size-edge cases (tests/debug_checks_run.py)
and reads the check records with hx_debug_checks.  Nothing is planted on the
GPU: a check that fires here is a planning or indexing bug.
"""

import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_debug_build_checks_stay_silent(gpu):
    env = dict(os.environ, HX_DEBUG="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "debug_checks_run.py")], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    rec = json.loads(r.stdout.strip().splitlines()[-1])
    assert rec["enabled"] is True
    assert rec["code"] == 0, (gpu.CHECK_NAMES.get(rec["code"]), rec)
    assert rec["results_ok"] is True


def test_release_build_reports_checks_off(gpu):
    enabled, code, a, b = gpu.hx_debug_checks()
    assert (enabled, code, a, b) == (gpu.DEBUG, 0, 0, 0)
