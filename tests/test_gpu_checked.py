"""The bounds-checked build (-DCDI_CHECKED) on odd shapes, every forward and adjoint tile and
a batch, against the oracle; and its check records a planted index.  Runs in a child process
(tests/checked_run.py) because one process must not load two builds of the library."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_runs_clean_and_records_a_planted_index():
    env = dict(os.environ, CDI_LIBRARY="checked")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checked_run.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and "checked ok" in r.stdout, (r.stdout[-2000:], r.stderr[-4000:])
