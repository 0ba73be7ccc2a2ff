"""The range-checked library build (every kernel array index checked; an
out-of-range one reported as TISSUE_E_BOUNDS instead of accessed) runs the
representative workloads of tests/_checked_run.py without a caught index and
with the oracle's results.  The stand-in for a memory sanitizer."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_runs_clean():
    env = dict(os.environ, TISSUE_CHECKED="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "_checked_run.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "checked build ok" in r.stdout
