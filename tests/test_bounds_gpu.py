"""The bounds-checked debug build (libwx_bounds.so, compiled with
WX_BOUNDS_CHECK): every guarded device access compares its element offset
with the size of its buffer, skips it when outside and reports it through
the context's status word (WX_ECUDA at the next synchronisation) -- the
stand-in for a memory checker, without a trap or a fault.  The grid paths
run on ragged and degenerate shapes under it in a child process (the
library is chosen when the binding loads) and must report nothing and still
match the oracle."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_grid_paths_report_no_out_of_bounds_access():
    from paper_1802_05839_gb300 import build
    if not os.path.exists(build.LIB_BOUNDS):
        build.build(bounds=True)
    env = dict(os.environ, WX_LIBRARY=build.LIB_BOUNDS)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "bounds_run.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    print(r.stdout[-3000:], r.stderr[-3000:])
    assert r.returncode == 0 and "BOUNDS_RUN_OK" in r.stdout
