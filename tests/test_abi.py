"""C-ABI checks that need no GPU: the library loads, exports every entry
point the header declares, and its host-only logic (spreading coefficients,
parameter validation, the create-time stability check) behaves."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import workloads
from paper_2409_16659_gb300 import mlswlbm as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(mlswlbm_\w+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    L = B.lib()
    names = _declared()
    assert "mlswlbm_create" in names and "mlswlbm_step" in names
    for name in sorted(names):
        assert hasattr(L, name), name
    assert names <= set(B.EXPORTS), names - set(B.EXPORTS)


def test_strerror_names_every_code():
    for code in range(0, -8, -1):
        assert B.mlswlbm_strerror(code) != "unknown error"
    assert B.mlswlbm_strerror(-99) == "unknown error"


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_spreading_from_tensions_matches_oracle(n):
    rng = np.random.default_rng(n)
    G = n + 2
    g = np.zeros((G, G))
    for a in range(G):
        for b in range(a + 1, G):
            g[a, b] = g[b, a] = rng.uniform(0.001, 0.05)
    S, gam = B.mlswlbm_spreading_from_tensions(n, g.ravel())
    So, gamo = oracle.spreading_from_tensions(dict(n=n, gamma=[0] * n, mu=[1] * n,
                                                   beta=[0] * n, nw=3, mw=2, hstar=0.1),
                                              g.ravel())
    assert gam == gamo
    for i in range(n):
        assert S[i] == So[i]


def test_check_params_accepts_workloads():
    assert B.mlswlbm_check_params(workloads.film2_d1q3_params()) == B.MLSW_OK
    assert B.mlswlbm_check_params(workloads.film3_d2q9_params()) == B.MLSW_OK


@pytest.mark.parametrize("mutate", [
    lambda p: p.update(n=0),
    lambda p: p.update(n=6, gamma=[0.01] * 6, mu=[1] * 6, beta=[1] * 6, S=None),
    lambda p: p.update(lattice=3),
    lambda p: p.update(nx=0),
    lambda p: p.update(tau=0.5),
    lambda p: p.update(tau=float("nan")),
    lambda p: p.update(hstar=0.0),
    lambda p: p.update(nw=2, mw=2),
    lambda p: p.update(nw=3, mw=0),
    lambda p: p.update(mu=[0.1, 0.0, 0.1]),
    lambda p: p.update(beta=[0.1, -1.0, 0.1]),
    lambda p: p.update(gamma=[0.01, float("inf"), 0.01]),
    lambda p: p.update(S=[[float("nan"), 0, 0], [0, 0], [0]]),
])
def test_check_params_rejects(mutate):
    p = workloads.film3_d2q9_params(8, 8)
    try:
        mutate(p)
        rc = B.mlswlbm_check_params(p)
    except ValueError:
        return  # rejected by the marshalling already
    assert rc == B.MLSW_ERR_ARG


def test_d1q3_needs_one_row():
    p = workloads.film2_d1q3_params(16)
    p["ny"] = 2
    assert B.mlswlbm_check_params(p) == B.MLSW_ERR_ARG


def _create_rc(p, h):
    s = B.make_params(p)
    a = np.ascontiguousarray(h, dtype=np.float32)
    out = ctypes.c_void_p()
    rc = B.lib().mlswlbm_create(ctypes.byref(s), a.ctypes.data_as(B._F), None,
                                ctypes.byref(out))
    if out:
        B.lib().mlswlbm_destroy(out)
    return rc, out


def test_create_rejects_bad_heights_on_host():
    p = workloads.film2_d1q3_params(16)
    h = np.ones((2, 1, 16))
    h[1, 0, 3] = np.nan
    rc, out = _create_rc(p, h)
    assert rc == B.MLSW_ERR_ARG and not out
    h[1, 0, 3] = -0.1
    rc, out = _create_rc(p, h)
    assert rc == B.MLSW_ERR_ARG and not out


def test_create_stability_check_rejects_no_slip_precursor():
    # no slip and a precursor of 0.07: friction -3 mu / h*^2 far below -2
    p = workloads.film3_d2q9_params(8, 8)
    p["beta"] = [0.0, 0.0, 0.0]
    h = workloads.film3_d2q9_heights(8, 8)
    rc, out = _create_rc(p, h)
    assert rc == B.MLSW_ERR_UNSTABLE and not out


def test_stability_check_can_be_skipped():
    p = workloads.film3_d2q9_params(8, 8)
    p["beta"] = [0.0, 0.0, 0.0]
    p["flags"] = B.MLSW_FLAG_SKIP_STABILITY_CHECK
    rc, out = _create_rc(p, workloads.film3_d2q9_heights(8, 8))
    # past the check; without a GPU the device set-up then fails cleanly
    assert rc in (B.MLSW_OK, B.MLSW_ERR_CUDA) and (rc == B.MLSW_OK) == bool(out)


def test_null_arguments():
    L = B.lib()
    assert L.mlswlbm_step(None, 1) == B.MLSW_ERR_ARG
    assert L.mlswlbm_get_heights(None, None) == B.MLSW_ERR_ARG
    assert L.mlswlbm_status(None) == B.MLSW_ERR_ARG
    assert L.mlswlbm_check_params(None) == B.MLSW_ERR_ARG
    assert L.mlswlbm_launch_count(None) == -1
    assert L.mlswlbm_max_abs_diff(None, None, 1, 1, None, None) == B.MLSW_ERR_ARG
    L.mlswlbm_destroy(None)


def test_gpu_test_cases_pass_the_stability_check():
    # the seeded parameter sets of the GPU parity tests must be accepted by
    # create (on this GPU-less host create then stops at the device set-up)
    from tests import test_gpu_parity as G
    import oracle as O
    cases = [G.one_step_case(*c) for c in G.ONE_STEP]
    cases = [(p, O.heights(p, f)) for p, f in cases]
    cases += [G.multistep_case(n) for n in G.MULTISTEP]
    cases += [G.edge_case(*c) for c in G.EDGE]
    for p, h in cases:
        rc, out = _create_rc(p, h)
        assert rc in (B.MLSW_OK, B.MLSW_ERR_CUDA), (rc, p)


def test_unet_argument_checks_and_parameter_count():
    """The U-Net's C entry points reject bad arguments before touching the
    GPU; its parameter count is that of the 15 convolutions of the four
    levels (32, 64, 128, 256 channels; 16 input planes, 16 outputs), 3 x 3
    taps plus a bias each."""
    import ctypes
    L = B.lib()
    convs = [(16, 32), (32, 32), (32, 64), (64, 64), (64, 128), (128, 128), (128, 256),
             (256, 256), (256 + 128, 128), (128, 128), (128 + 64, 64), (64, 64),
             (64 + 32, 32), (32, 32), (32, 16)]
    assert L.mlswlbm_unet_param_count() == sum(9 * ci * co + co for ci, co in convs)
    out = ctypes.c_void_p(1)
    ex = (ctypes.c_double * 16)(*([0.5] * 16))
    nan = (ctypes.c_double * 1)(float("nan"))
    for args, want in [((0, 256, 256, 4, 0, None), B.MLSW_ERR_ARG),
                       ((6, 256, 256, 4, 0, None), B.MLSW_ERR_ARG),
                       ((3, 256, 256, 0, 0, None), B.MLSW_ERR_ARG),
                       ((3, 256, 256, 4, 14, ex), B.MLSW_ERR_ARG),
                       ((3, 256, 256, 4, 2, None), B.MLSW_ERR_ARG),
                       ((3, 256, 256, 4, 1, nan), B.MLSW_ERR_ARG),
                       ((3, 192, 256, 4, 0, None), B.MLSW_ERR_UNSUPPORTED),
                       ((3, 256, 64, 4, 0, None), B.MLSW_ERR_UNSUPPORTED),
                       ((3, 8192, 256, 4, 0, None), B.MLSW_ERR_UNSUPPORTED)]:
        rc = L.mlswlbm_unet_create(*args, 1, 1.0, 4.0, None, ctypes.byref(out))
        assert rc == want and not out.value, (args[:5], rc)
        out = ctypes.c_void_p(1)
    for scales in [(0.0, 4.0), (1.0, -1.0), (float("inf"), 4.0)]:
        rc = L.mlswlbm_unet_create(3, 256, 256, 4, 0, None, 1, *scales, None, ctypes.byref(out))
        assert rc == B.MLSW_ERR_ARG, scales
    assert L.mlswlbm_unet_create(3, 256, 256, 4, 0, None, 1, 1.0, 4.0, None, None) == B.MLSW_ERR_ARG
    assert L.mlswlbm_unet_predict(None, None, None, 1) == B.MLSW_ERR_ARG
    assert L.mlswlbm_unet_train_step(None, None, None, 1, 1e-3, None) == B.MLSW_ERR_ARG
    L.mlswlbm_unet_destroy(None)


def test_audit_error_and_many_instance_calls_reject_bad_arguments():
    """mlswlbm_max_abs_diff and the many-instance batch height calls check
    their arguments on the host before any device work (and the Python
    binding checks tensor types and index ranges before calling them)."""
    import ctypes
    import torch
    L = B.lib()
    p = ctypes.c_void_p(16)
    assert L.mlswlbm_max_abs_diff(None, p, 1, 1, p, None) == B.MLSW_ERR_ARG
    assert L.mlswlbm_max_abs_diff(p, p, 0, 1, p, None) == B.MLSW_ERR_ARG
    assert L.mlswlbm_max_abs_diff(p, p, 1, 0, p, None) == B.MLSW_ERR_ARG
    idx = (ctypes.c_int * 1)(0)
    for fn in (L.mlswlbm_batch_get_heights_device_many, L.mlswlbm_batch_set_heights_device_many):
        assert fn(None, 1, idx, p) == B.MLSW_ERR_ARG
    with pytest.raises(ValueError):  # host tensors
        B.max_abs_diff(torch.zeros(2, 3), torch.zeros(2, 3))
    fake = B.Batch.__new__(B.Batch)  # the index check needs only the shapes
    fake.shapes = [(3, 8, 8), (2, 4, 4)]
    with pytest.raises(ValueError):
        fake._many([0, 2], None)
    with pytest.raises(ValueError):
        fake._many([-1], None)
