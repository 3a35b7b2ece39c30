"""Batches of independent D2Q9 lattices (mlswlbm_batch_*).

Every instance of a batch runs the single-lattice step's arithmetic: with
the same tile height its heights equal those of mlswlbm_create/step bit for
bit; with the other tile height (one cell per thread instead of a packed
FP32x2 pair, where the compiler may contract a multiply-add differently) they
agree to FP32 rounding. The device mode amplitudes are checked against an
FFT of the read-back heights, and a single-mode perturbation against the
independently linearised step G(q) of tests/lsa.py (the linear-stability
pin): the batched stability sweep measures growth rates this way.
"""
import numpy as np
import pytest

import workloads
from paper_2409_16659_gb300 import mlswlbm as B
from tests import lsa

pytestmark = pytest.mark.gpu


def _mixed_instances():
    """Mixed layer counts, sizes (ragged too), kernel modes and parameters."""
    out = []
    p = workloads.film3_d2q9_params(64, 96)
    out.append((p, workloads.film3_d2q9_heights(64, 96, seed=5)))           # n = 3, fast mode
    for seed, n, nx, ny, tau in [(11, 2, 64, 64, 1.0), (12, 4, 72, 40, 1.0),
                                 (13, 5, 64, 64, 0.9), (14, 3, 40, 72, 1.2),
                                 (15, 1, 96, 32, 1.0), (16, 2, 33, 17, 1.0)]:
        p = workloads.random_params(seed, n, B.MLSW_D2Q9, nx, ny, tau=tau)
        out.append((p, workloads.random_heights(100 + seed, p)))
    # on a corrugated substrate
    p = dict(workloads.random_params(17, 3, B.MLSW_D2Q9, 48, 32), sub_amp=0.1, sub_kx=2, sub_ky=1)
    out.append((p, workloads.random_heights(117, p)))
    # with the exponential (charged-surface) wetting potential
    p = workloads.random_params(18, 2, B.MLSW_D2Q9, 40, 40)
    p.update(wet_kind=1, kappa=1.0 / p["hstar"])
    out.append((p, workloads.random_heights(118, p)))
    return out


def _single(p, h, steps):
    with B.Solver(p, h) as s:
        s.step(steps)
        return s.get_heights()


def test_batch_matches_single_solver_bit_exact():
    inst = _mixed_instances()
    with B.Batch([p for p, _ in inst], [h for _, h in inst]) as b:
        assert b.groups() >= 4
        b.step(30)
        for j, (p, h) in enumerate(inst):
            assert b.tile_rows(j) == (16 if p["n"] <= 3 else 8)
            assert np.array_equal(b.get_heights(j), _single(p, h, 30)), j
        assert b.status() == B.MLSW_OK
        # every step is one launch, whatever the number of groups
        n0 = b.launch_count()
        b.step(3)
        assert b.launch_count() - n0 == 3


def test_batch_eight_row_tiles_agree_to_fp32_rounding():
    inst = _mixed_instances()
    with B.Batch([p for p, _ in inst], [h for _, h in inst], flags=B.MLSW_BATCH_TILE8) as b:
        b.step(30)
        for j, (p, h) in enumerate(inst):
            assert b.tile_rows(j) == 8
            ref = _single(p, h, 30).astype(np.float64)
            got = b.get_heights(j).astype(np.float64)
            assert np.abs(got - ref).max() <= 2e-6 * np.abs(ref).max(), j


def test_batch_autotune_chooses_a_tile_height_and_restores_the_state():
    inst = _mixed_instances()
    with B.Batch([p for p, _ in inst], [h for _, h in inst], flags=B.MLSW_BATCH_AUTOTUNE) as b:
        for j, (p, h) in enumerate(inst):
            assert b.tile_rows(j) in ((8, 16) if p["n"] <= 3 else (8,))
            # the timing steps are undone: the state is f_eq(h_init) again
            np.testing.assert_allclose(b.get_heights(j), np.asarray(h, dtype=np.float32),
                                       rtol=0, atol=1e-6)
        b.step(10)
        for j, (p, h) in enumerate(inst):
            ref = _single(p, h, 10).astype(np.float64)
            got = b.get_heights(j).astype(np.float64)
            assert np.abs(got - ref).max() <= 2e-6 * np.abs(ref).max(), j


def test_batch_modes_match_fft_of_heights():
    inst = _mixed_instances()
    rng = np.random.default_rng(3)
    kx = rng.integers(-5, 6, len(inst))
    ky = rng.integers(-5, 6, len(inst))
    with B.Batch([p for p, _ in inst], [h for _, h in inst]) as b:
        b.step(20)
        m = b.modes(kx, ky)
        for j, (p, h) in enumerate(inst):
            hh = b.get_heights(j).astype(np.float64)
            F = np.fft.fft2(hh, axes=(1, 2))
            n, ny, nx = hh.shape
            want = F[:, int(ky[j]) % ny, int(kx[j]) % nx]
            scale = np.abs(hh).sum(axis=(1, 2))
            assert np.all(np.abs(m[j, :n] - want) <= 1e-6 * scale), j
            assert np.all(m[j, n:] == 0)


@pytest.mark.parametrize("seed,n,mode", [(21, 2, (1, 0)), (22, 3, (2, 1)), (23, 2, (0, 3))])
def test_single_mode_follows_linearised_step_in_a_batch(seed, n, mode):
    """A 1e-4 single-mode perturbation of a flat film, stepped 2000 times in
    a batch, follows G(q)^t of the linearised scheme: the sweep's growth-rate
    measurement."""
    side = 64
    p = workloads.random_params(seed, n, B.MLSW_D2Q9, side, side, tau=1.0, multilayer_S=False)
    rng = np.random.default_rng(seed)
    h0 = rng.uniform(0.6, 1.1, n)
    amps = rng.uniform(-1, 1, n)
    eps = 1e-4
    h = workloads.single_mode_heights(p, h0, amps, mode, eps)
    q = (2 * np.pi * mode[0] / side, 2 * np.pi * mode[1] / side)
    G = lsa.step_matrix(p, h0, q)
    Q = 9
    v = np.zeros(n * Q, dtype=complex)
    v[0::Q] = eps * amps / 2  # f_0 carries h at rest; cos -> half at +q
    others = workloads.film3_d2q9_params(64, 64)  # a second instance in the batch
    with B.Batch([p, others], [h, workloads.film3_d2q9_heights(64, 64)]) as b:
        done = 0
        for t in (500, 1000, 2000):
            b.step(t - done)
            done = t
            got = b.modes([mode[0], 0], [mode[1], 0])[0, :n] / side ** 2
            want = (np.linalg.matrix_power(G, t) @ v).reshape(n, Q).sum(axis=1)
            assert np.abs(got - want).max() <= 2e-3 * np.abs(want).max() + 1e-9, (t, got, want)


def test_full_size_stability_sweep_sampled_against_oracle():
    """The 512-instance stability sweep of the bench in its launch
    configuration (autotuned tile heights, the step replayed as a CUDA
    graph): after 20 steps, the smallest and the largest instance of every
    layer count equal the FP64 oracle to 1e-5 of their largest height."""
    import oracle
    inst = workloads.sweep_instances()
    picks = []
    for n in (2, 3, 4, 5):
        js = [j for j, (p, *_r) in enumerate(inst) if p["n"] == n]
        picks.append(min(js, key=lambda j: inst[j][0]["nx"]))
        picks.append(max(js, key=lambda j: inst[j][0]["nx"]))
    with B.Batch([p for p, *_r in inst], [h for _p, h, *_r in inst],
                 flags=B.MLSW_BATCH_AUTOTUNE) as b:
        b.step(20)
        assert b.status() == B.MLSW_OK
        for j in picks:
            p, h0 = inst[j][0], inst[j][1]
            hg = b.get_heights(j).astype(np.float64)
            f = oracle.run(p, oracle.init(p, h0.astype(np.float64).ravel()), 20)
            hr = oracle.heights(p, f).reshape(hg.shape)
            assert np.abs(hg - hr).max() <= 1e-5 * np.abs(hr).max(), (j, p["n"], p["nx"])


def test_selected_instances_step_and_the_others_keep_their_state():
    """mlswlbm_batch_select: over odd and even step counts, each instance
    ends after exactly the steps it was selected for, bit for bit as a
    single solver; one left out keeps its state (heights and modes), and a
    restart from new heights while left out takes effect when selected."""
    inst = _mixed_instances()[:5]
    P, H = [p for p, _ in inst], [h for _, h in inst]
    import torch
    with B.Batch(P, H) as b, B.Batch(P, H) as fresh:
        kx = np.ones(len(P), dtype=np.int32)
        ky = np.zeros(len(P), dtype=np.int32)
        m_init = fresh.modes(kx, ky)
        steps = np.zeros(len(P), dtype=int)
        for sel, k in (([0, 2], 7), ([1, 2, 4], 5), ([], 3), ([3], 1)):
            b.select(sel)
            b.step(k)
            steps[sel] += k
        # instance 1 and 4 have been left out over an odd number of steps
        m = b.modes(kx, ky)
        for j in range(len(P)):
            if steps[j] == 0:
                assert np.array_equal(m[j], m_init[j]), j
        for j, (p, h) in enumerate(inst):
            assert np.array_equal(b.get_heights(j), _single(p, h, int(steps[j]))), (j, steps[j])
        # restart a left-out instance from other heights, then step everyone
        h2 = workloads.random_heights(999, P[3]).astype(np.float32)
        b.set_heights_device(3, torch.from_numpy(h2).cuda())
        b.select(range(len(P)))
        b.step(4)
        for j, (p, h) in enumerate(inst):
            if j == 3:
                # a restart keeps the rest-population shift of create, as
                # the single solver's mlswlbm_set_heights does
                with B.Solver(p, h) as s:
                    s.set_heights(h2)
                    s.step(4)
                    want = s.get_heights()
            else:
                want = _single(p, h, int(steps[j]) + 4)
            assert np.array_equal(b.get_heights(j), want), j
        assert b.status() == B.MLSW_OK
    with B.Batch(P, H) as b:
        ip = np.array([0, 0], dtype=np.int32)
        assert B.lib().mlswlbm_batch_select(b._b, 2, ip.ctypes.data_as(
            B.ctypes.POINTER(B.ctypes.c_int))) == B.MLSW_ERR_ARG


def test_device_heights_of_many_instances_at_once():
    """mlswlbm_batch_get/set_heights_device_many equal the one-instance calls
    (any order of indices), and reject an index out of range."""
    import torch
    inst = _mixed_instances()
    with B.Batch([p for p, _ in inst], [h for _, h in inst]) as b:
        b.step(7)
        order = [3, 0, 5, 2]
        sizes = [int(np.prod(b.shapes[j])) for j in order]
        many = torch.empty(sum(sizes), dtype=torch.float32, device="cuda")
        b.get_heights_device_many(order, many)
        off = 0
        for j, sz in zip(order, sizes):
            one = torch.empty(sz, dtype=torch.float32, device="cuda")
            b.get_heights_device(j, one)
            assert torch.equal(many[off:off + sz], one), j
            off += sz
        # restart the listed instances from their own heights: both calls
        # give the same states, so the next steps give the same heights
        b.set_heights_device_many(order, many)
        b.step(3)
        got = [b.get_heights(j) for j in order]
    with B.Batch([p for p, _ in inst], [h for _, h in inst]) as c:
        c.step(7)
        off = 0
        for j, sz in zip(order, sizes):
            one = torch.empty(sz, dtype=torch.float32, device="cuda")
            c.get_heights_device(j, one)
            c.set_heights_device(j, one)
        c.step(3)
        for j, g in zip(order, got):
            assert np.array_equal(c.get_heights(j), g), j
        with pytest.raises(ValueError):
            c.get_heights_device_many([len(inst)], torch.empty(1, device="cuda"))
        import ctypes
        bad = (ctypes.c_int * 1)(len(inst))
        assert B.lib().mlswlbm_batch_get_heights_device_many(
            c._b, 1, bad, ctypes.c_void_p(many.data_ptr())) == B.MLSW_ERR_ARG
