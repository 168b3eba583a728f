"""The bounds-checked build (libwilson_checked.so: every internal site index
tested against its array, violations recorded instead of trapping) runs the
library's kernels -- every operator, precision and hop variant on tiny and
odd lattices, the solvers in each mode, the multi-shift solver and the
backward -- without recording an out-of-range index.  It stands in for a
memory checker, which this GPU pool does not offer.  The pass runs in a
process of its own (tests/checked_battery.py) because a process loads one
build of the library."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_records_no_out_of_range_index():
    env = dict(os.environ, WL_LIBRARY="checked")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checked_battery.py")], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["checked_build"] and line["first_violation"] == 0 and line["calls"] > 100, line
