"""The bounds-checked build of the library (-DMLSW_DEBUG) on tiny lattices.

That build checks every padded-layout index, every shared-memory access and
global store of the step kernels and the coordinates of every tile copy; an
access out of range is counted (mlswlbm_debug_bounds_violations) and sent to
a padding cell instead of faulting. It stands in for a memory checker. The
test builds it, runs it in a child process (the parent keeps the release
library loaded) on lattices from 1 x 1 to 8 x 8 cells and one of several
ragged tiles, n = 1..5 on both lattices, and asks for two things: no access
out of range, and heights within 1e-5 of the FP64 oracle after 20 steps
(the paper's step, Eq. BGK), which is the parity bar of the release build.
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.gpu

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, %(root)r)
import oracle, workloads
from paper_2409_16659_gb300 import mlswlbm as B
B.LIB_PATH = %(lib)r
cases = []
for n in (1, 2, 3, 4, 5):
    for nx, ny in ((1, 1), (2, 3), (3, 2), (4, 4), (5, 7), (8, 8), (37, 21)):
        cases.append((n, 2, nx, ny, 1.0))
    cases.append((n, 2, 6, 5, 0.8))
    for nx in (1, 2, 3, 5, 8, 130):
        cases.append((n, 1, nx, 1, 1.0))
out = []
for n, lat, nx, ny, tau in cases:
    p = workloads.random_params(500 + 7 * n + nx + 3 * ny, n, lat, nx, ny, tau=tau)
    h0 = np.asarray(workloads.random_heights(600 + n + nx, p, 0.5, 1.0, 5e-3), np.float32)
    with B.Solver(p, h0) as s:
        s.step(20)
        hg = s.get_heights().astype(np.float64)
        st = s.status()
    f = oracle.run(p, oracle.init(p, h0.astype(np.float64).ravel()), 20)
    hr = oracle.heights(p, f)
    err = float(np.abs(hg - hr).max() / np.abs(hr).max())
    out.append({"case": [n, lat, nx, ny, tau], "err": err, "status": int(st),
                "violations": B.mlswlbm_debug_bounds_violations()})
print(json.dumps(out))
"""


def test_bounds_checked_build_on_tiny_lattices():
    from paper_2409_16659_gb300 import _build, mlswlbm as B
    # the release library the other tests load reports that it is not this build
    assert B.mlswlbm_debug_bounds_violations() is None
    lib = _build.build(debug=True)
    r = subprocess.run([sys.executable, "-c", CHILD % {"root": ROOT, "lib": lib}],
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert len(res) == 5 * 14
    for c in res:
        assert c["violations"] == 0, c
        assert c["status"] == B.MLSW_OK, c
        assert c["err"] <= 1e-5, c
