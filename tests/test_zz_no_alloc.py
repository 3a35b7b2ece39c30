"""mlswlbm_diagnostics_noalloc: diagnostics for callers that cannot allocate.

Callers whose device memory is held by a pool allocator, or whose loops
cannot afford the device-wide synchronisation of cudaMalloc / cudaFree, use
this entry point; it takes a caller-owned population array and keeps its
scratch in a static device array of the library. This file is collected
last, so a run that stops at the first failure has run every other test.
The check: through the C ABI, two calls in a row agree with
mlswlbm_get_diagnostics of a handle holding the same state, within the
tolerances the diagnostics tests use (mass and min h 1e-6, kinetic energy
1e-4, relative).
"""
import numpy as np
import pytest

import workloads
from paper_2409_16659_gb300 import mlswlbm as B

pytestmark = pytest.mark.gpu


def _close(got, want, n):
    np.testing.assert_allclose(got[:n], want[0], rtol=1e-6)
    assert got[n] == pytest.approx(want[1], rel=1e-4)
    assert got[n + 1] == pytest.approx(want[2], rel=1e-6)


@pytest.mark.parametrize("lat", [2, 1])
def test_noalloc_diagnostics_match_handle_diagnostics_twice(lat):
    import torch
    if lat == 2:
        p = workloads.film3_d2q9_params(300, 170)
    else:
        p = workloads.film2_d1q3_params(4099)
    n = p["n"]
    f = workloads.random_populations(31, p, 0.5, 1.0, 2e-3).astype(np.float32)
    with B.Solver(p, f.sum(axis=1)) as s:
        s.set_state(f)
        s.step(7)
        want = s.get_diagnostics()
        f_true = s.get_state()
        H, g = s.save_state()
    # true populations (H = NULL), then the internal representation with H
    ft = torch.from_numpy(f_true.reshape(-1)).cuda()
    fg = torch.from_numpy(g.reshape(-1)).cuda()
    out = torch.empty(n + 2, dtype=torch.float64, device="cuda")
    for _ in range(2):
        B.mlswlbm_diagnostics_noalloc(p, ft, out)
        torch.cuda.synchronize()
        _close(out.cpu().numpy(), want, n)
        out.fill_(np.nan)
        B.mlswlbm_diagnostics_noalloc(p, fg, out, H=H)
        torch.cuda.synchronize()
        _close(out.cpu().numpy(), want, n)
        out.fill_(np.nan)


def test_noalloc_rejects_lattices_beyond_the_static_scratch():
    import torch
    p = workloads.film3_d2q9_params(8192, 8193)  # 8192 * 8193 > 4096 * 16384 cells
    f = torch.zeros(16, dtype=torch.float32, device="cuda")
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    rc = B.lib().mlswlbm_diagnostics_noalloc(
        B.ctypes.byref(B.make_params(p)), B.ctypes.c_void_p(f.data_ptr()), None,
        B.ctypes.c_void_p(out.data_ptr()), None)
    assert rc == B.MLSW_ERR_UNSUPPORTED
