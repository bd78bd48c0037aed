"""The debug build (device-side checks instead of the closed sanitizer): in a
separate process that loads libdgw_debug.so, valid inputs raise no fault and
give the release results (parity with the oracle), and a NaN planted in one
node of the input state -- a valid address holding an invalid value -- is
reported with its element, once, while the kernel carries on."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import sys
sys.path.insert(0, sys.argv[1]); sys.path.insert(0, sys.argv[1] + "/tests")
import numpy as np, torch
from paper_1711_01175_gb300 import build, capi
build.build(debug=True)
assert capi.load()._name.endswith("libdgw_debug.so"), capi.load()._name
from harness import Case, FP64_TOL, assert_parity
c = Case(3, 3, 0.1, material=2, seed=8)
u = c.u0.copy()
assert_parity(c.gpu_rhs(u), c.op.rhs(u), FP64_TOL)
st, code, el, cnt = capi.dgw_debug_status(c.solver._ctx)
assert st == 0 and code == 0 and cnt == 0, (st, code, el, cnt)
u[4, 13, 17] = np.nan
c.gpu_rhs(u)
st, code, el, cnt = capi.dgw_debug_status(c.solver._ctx)
assert st == 0 and code == 1 and el == 13 and cnt == 1, (st, code, el, cnt)
st, code, el, cnt = capi.dgw_debug_status(c.solver._ctx)          # cleared by the read
assert code == 0 and cnt == 0
print("debug checks ok")
'''


def test_debug_build_reports_a_planted_nan_and_nothing_else():
    env = dict(os.environ, DGW_DEBUG_CHECKS="1")
    r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    assert "debug checks ok" in r.stdout


def test_release_build_has_no_debug_status():
    from paper_1711_01175_gb300 import Solver, capi
    import __graft_entry__ as g
    g.build()
    s = Solver(2)
    st, _, _, _ = capi.dgw_debug_status(s._ctx)
    assert st == -7 and "DGW_DEBUG_CHECKS" in capi.dgw_last_error(s._ctx)
    s.close()
