"""The U-Net workflow on the GPU: trajectories read on the device, and the
rollout judged by the LBM (surrogate.judged_rollout) in its two limits.

- A bound no window can meet: every instance fails its first audit, goes
  back to its start and finishes on the LBM alone. The result must equal the
  batched solver's bit for bit: a solver restarted at rest from the initial
  heights is the batch instance's own start, and a batch instance steps
  with exactly the single solver's arithmetic.
- No bound: every window passes. The surrogate keeps each layer's mass by
  construction and the LBM conserves it, so per-layer mass must hold to
  FP32 round-off (1e-6 relative) over the whole rollout.
"""
import numpy as np
import pytest

import workloads
from paper_2409_16659_gb300 import mlswlbm as B
from paper_2409_16659_gb300 import surrogate as S

pytestmark = pytest.mark.gpu

SIDE, M, WINDOWS = 128, 4, 4


def _case():
    params = [workloads.film3_d2q9_params(SIDE, SIDE) for _ in range(M)]
    heights = [np.asarray(workloads.film3_d2q9_heights(SIDE, SIDE, seed=700 + j), np.float32)
               for j in range(M)]
    return params, heights


def test_device_trajectories_equal_host_trajectories():
    params, heights = _case()
    a = S.trajectories(params, heights, 2)
    b = S.trajectories_device(params, heights, 2)
    assert np.array_equal(a.cpu().numpy(), b.cpu().numpy())


def test_failed_audits_fall_back_to_the_lbm_exactly():
    params, heights = _case()
    with B.UNet(3, SIDE, SIDE, 2, seed=1) as u:
        h, st = S.judged_rollout(u, params, heights, WINDOWS, audit_every=2, bound=0.0)
    ref, _ = S.lbm_batched(params, heights, WINDOWS)
    assert st["fallback_instances"] == M and st["surrogate_windows"] == 0
    assert np.array_equal(h.cpu().numpy(), ref.cpu().numpy())
    per, _ = S.lbm_per_instance(params, heights, WINDOWS)
    assert np.array_equal(per.cpu().numpy(), ref.cpu().numpy())


def test_accepted_windows_keep_every_layer_mass():
    params, heights = _case()
    with B.UNet(3, SIDE, SIDE, 2, seed=1) as u:
        h, st = S.judged_rollout(u, params, heights, WINDOWS, audit_every=2, bound=np.inf)
    assert st["fallback_instances"] == 0
    # windows 0, 1 and 3 are audited (the first, every second, the last)
    assert st["audited_windows"] == M * 3
    assert st["surrogate_windows"] == M * 1
    m0 = np.array([x.astype(np.float64).sum(axis=(1, 2)) for x in heights])
    m1 = h.double().sum(dim=(2, 3)).cpu().numpy()
    np.testing.assert_allclose(m1, m0, rtol=1e-6)


def test_max_abs_diff_is_the_windows_height_error():
    """mlswlbm_max_abs_diff, the audit's error, against numpy: float4 and
    scalar paths (item sizes divisible by 4 or not, an unaligned start),
    more items than one grid row holds, and a non-finite difference, which
    must count as +inf so that a non-finite prediction fails any bound."""
    import torch
    rng = np.random.default_rng(5)

    def check(a, b):
        got = B.max_abs_diff(a, b).cpu().numpy()
        an, bn = a.cpu().numpy(), b.cpu().numpy()
        want = np.abs(an - bn).reshape(an.shape[0], -1).max(axis=1)
        want = np.where(np.isfinite(want), want, np.inf).astype(np.float32)
        assert np.array_equal(got, want)

    for shape in [(5, 3, 64, 64), (3, 7, 5), (1, 1), (70000, 4)]:
        a = torch.from_numpy(rng.normal(size=shape).astype(np.float32)).cuda()
        b = torch.from_numpy(rng.normal(size=shape).astype(np.float32)).cuda()
        check(a, b)
    # an item starting off the 16-byte boundary takes the scalar path
    base = torch.from_numpy(rng.normal(size=4 * 1024 + 1).astype(np.float32)).cuda()
    other = torch.from_numpy(rng.normal(size=4 * 1024).astype(np.float32)).cuda()
    check(base[1:].view(4, 1024), other.view(4, 1024))
    # NaN and inf in item 1 only; equal items give exactly 0
    a = torch.from_numpy(rng.normal(size=(3, 2, 16, 16)).astype(np.float32)).cuda()
    b = a.clone()
    b[1, 0, 3, 4] = float("nan")
    b[1, 1, 0, 0] = float("inf")
    got = B.max_abs_diff(a, b).cpu().numpy()
    assert got[0] == 0.0 and got[2] == 0.0 and np.isposinf(got[1])
    with pytest.raises(ValueError):
        B.max_abs_diff(a, b[:2].contiguous())
