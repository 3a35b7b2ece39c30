"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (FP32 device arithmetic vs FP64 oracle, unit round-off
u = 2^-24 ~ 6e-8):
  * heights after many steps: max |h_gpu - h_ref| / max |h_ref| <= 1e-5, the
    target the solver is specified to;
  * one step from a given state: every population within 4e-6 * max h. A
    population is formed from O(50) FP32 operations on O(h) quantities,
    each contributing at most u * h, and the pressure forces are O(1e-2 h);
  * friction of independent cells: 1e-4 of the largest |R| of the cell, the
    FP32 elimination error bound cond(L) * u with cond(L) <= ~1e3 for the
    thicknesses drawn here;
  * invariants that the kernels keep exactly (flat film, translation,
    checkpoint) are compared bit for bit.
"""
import numpy as np
import pytest

import json
import os

import oracle
import workloads
from paper_2409_16659_gb300 import mlswlbm as B
from tests import droplets, lsa

pytestmark = pytest.mark.gpu


def _f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def _run_both(p, h0, steps):
    h0 = _f32(h0)
    with B.Solver(p, h0) as s:
        s.step(steps)
        hg = s.get_heights().astype(np.float64)
    f = oracle.run(p, oracle.init(p, h0.ravel()), steps)
    return hg, oracle.heights(p, f)


def _relmax(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def test_film2_d1q3_512_cells_1000_steps():
    p = workloads.film2_d1q3_params(512)
    hg, hr = _run_both(p, workloads.film2_d1q3_heights(512), 1000)
    assert _relmax(hg, hr) <= 1e-5


def test_film2_d1q3_512_cells_10000_steps():
    """The two-layer D1Q3 film at its full length, 10 000 steps (one
    persistent launch on the GPU): heights within 1e-5 of the oracle's."""
    p = workloads.film2_d1q3_params(512)
    h0 = workloads.film2_d1q3_heights(512)
    hg, hr = _run_both(p, h0, 10000)
    assert _relmax(hg, hr) <= 1e-5


def test_film3_d2q9_ragged_1000_steps():
    # 72 x 40 cells: 3 x 3 tiles of 32 x 16, ragged in both directions
    p = workloads.film3_d2q9_params(72, 40)
    hg, hr = _run_both(p, workloads.film3_d2q9_heights(72, 40), 1000)
    assert _relmax(hg, hr) <= 1e-5


def test_film3_d2q9_128_1000_steps():
    """The three-layer spinodal film's parameters (the 1024^2 benchmark
    recipe) on 128 x 128 cells, 1000 steps through mlswlbm_create / step /
    get_heights: every height within 1e-5 of the FP64 oracle's, relative to
    the largest height (Eq. BGK with the lattice of the LBM section)."""
    p = workloads.film3_d2q9_params(128, 128)
    hg, hr = _run_both(p, workloads.film3_d2q9_heights(128, 128, seed=2), 1000)
    assert _relmax(hg, hr) <= 1e-5
    # the film has moved away from its start by far more than the tolerance
    h0 = _f32(workloads.film3_d2q9_heights(128, 128, seed=2)).reshape(hr.shape)
    assert np.abs(hr - h0).max() > 1e-4


# -- the seeded cases (also checked on the CPU for create-time stability) ----
ONE_STEP = [(n, lat, tau) for n in (1, 2, 3, 4, 5)
            for lat, tau in ((2, 1.0), (2, 0.8), (1, 1.0), (1, 1.4))]
MULTISTEP = [2, 4, 5]
EDGE = [(2, 1, 1), (2, 2, 3), (2, 1, 7), (2, 5, 1), (2, 33, 17),
        (1, 1, 1), (1, 2, 1), (1, 3, 1), (1, 129, 1)]


def one_step_case(n, lat, tau):
    nx, ny = (37, 21) if lat == 2 else (301, 1)
    p = workloads.random_params(40 + n, n, lat, nx, ny, tau=tau)
    return p, _f32(workloads.random_populations(50 + n, p, 0.5, 1.0, 2e-3))


def multistep_case(n):
    p = workloads.random_params(70 + n, n, 2, 45, 33)
    return p, workloads.random_heights(80 + n, p, 0.5, 1.1, 2e-3)


def edge_case(lat, nx, ny):
    p = workloads.random_params(90 + nx + ny, 3, lat, nx, ny)
    return p, workloads.random_heights(91 + nx, p, 0.6, 1.0, 5e-3)


@pytest.mark.parametrize("n,lat,tau", ONE_STEP)
def test_one_step_from_random_state(n, lat, tau):
    p, f = one_step_case(n, lat, tau)
    hmax = oracle.heights(p, f).max()
    with B.Solver(p, oracle.heights(p, f)) as s:
        s.set_state(f)
        s.step(1)
        fg = s.get_state().astype(np.float64)
        assert s.status() == B.MLSW_OK
    fr = oracle.step(p, f)
    assert np.abs(fg - fr).max() <= 4e-6 * hmax


@pytest.mark.parametrize("n", MULTISTEP)
def test_random_params_multistep(n):
    p, h0 = multistep_case(n)
    hg, hr = _run_both(p, h0, 300)
    assert _relmax(hg, hr) <= 1e-5


# the exponential (charged-surface) wetting potential, decay length h*:
# every layer count, both lattices, tau = 1 and tau != 1
EXP_ONE_STEP = [(n, lat, tau) for n in (1, 2, 3, 5) for lat, tau in ((2, 1.0), (2, 0.8), (1, 1.0))]


@pytest.mark.parametrize("n,lat,tau", EXP_ONE_STEP)
def test_one_step_with_the_exponential_potential(n, lat, tau):
    p, f = one_step_case(n, lat, tau)
    p = dict(p, wet_kind=1, kappa=1.0 / p["hstar"])
    hmax = oracle.heights(p, f).max()
    with B.Solver(p, oracle.heights(p, f)) as s:
        s.set_state(f)
        s.step(1)
        fg = s.get_state().astype(np.float64)
        assert s.status() == B.MLSW_OK
    fr = oracle.step(p, f)
    assert np.abs(fg - fr).max() <= 4e-6 * hmax


def test_exponential_potential_multistep_and_free_energy():
    p, h0 = multistep_case(3)
    p = dict(p, wet_kind=1, kappa=1.0 / p["hstar"])
    hg, hr = _run_both(p, h0, 300)
    assert _relmax(hg, hr) <= 1e-5
    # the power law ends 7e-5 away: the bound above tells the two forms apart
    q = dict(p, wet_kind=0)
    hp = oracle.heights(q, oracle.run(q, oracle.init(q, _f32(h0).ravel()), 300))
    assert _relmax(hp.reshape(hr.shape), hr) > 3e-5
    with B.Solver(p, h0) as s:
        s.step(50)
        F = s.free_energy()
        want = droplets.free_energy(p, s.get_heights().astype(np.float64))
    assert F == pytest.approx(want, rel=1e-10, abs=1e-12)


@pytest.mark.parametrize("lat,nx,ny", EDGE)
def test_degenerate_and_edge_sizes(lat, nx, ny):
    p, h0 = edge_case(lat, nx, ny)
    hg, hr = _run_both(p, h0, 25)
    assert _relmax(hg, hr) <= 1e-5


def test_flat_film_stays_bit_exact():
    p = workloads.film3_d2q9_params(50, 30)
    h0 = np.broadcast_to(np.array([1.0, 0.8, 0.6])[:, None, None], (3, 30, 50)).copy()
    with B.Solver(p, h0) as s:
        f0 = s.get_state()
        s.step(200)
        assert np.array_equal(s.get_state(), f0)


def test_mass_conserved_to_fp32_roundoff():
    p = workloads.film3_d2q9_params(128, 96)
    h0 = _f32(workloads.film3_d2q9_heights(128, 96))
    with B.Solver(p, h0) as s:
        m0, _, _ = s.get_diagnostics()
        s.step(2000)
        m1, ke, hmin = s.get_diagnostics()
    np.testing.assert_allclose(m0, h0.sum(axis=(1, 2)), rtol=1e-12)
    assert np.abs(m1 - m0).max() / m0.max() <= 1e-6
    assert hmin > 0.5 and np.isfinite(ke)


def test_translation_equivariance_bit_exact():
    p = workloads.film3_d2q9_params(70, 36)
    h0 = workloads.film3_d2q9_heights(70, 36)
    hs = np.roll(h0, (5, -11), axis=(1, 2))
    with B.Solver(p, h0) as a, B.Solver(p, hs) as b:
        a.step(20)
        b.step(20)
        assert np.array_equal(np.roll(a.get_heights(), (5, -11), axis=(1, 2)), b.get_heights())


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_friction_eval_matches_oracle(n):
    import torch
    rng = np.random.default_rng(200 + n)
    ncell = 257
    p = workloads.random_params(300 + n, n, 2, 1, 1)
    p["beta"] = list(rng.uniform(0.0, 1.5, n))
    p["beta"][0] = 0.0 if n % 2 else p["beta"][0]
    h = rng.uniform(0.06, 1.5, (n, ncell)).astype(np.float32)
    Jx = rng.normal(0, 1e-3, (n, ncell)).astype(np.float32)
    Jy = rng.normal(0, 1e-3, (n, ncell)).astype(np.float32)
    dev = lambda a: torch.from_numpy(a).cuda().contiguous()
    Rx, Ry = B.mlswlbm_friction_eval(p, dev(h), dev(Jx), dev(Jy))
    torch.cuda.synchronize()
    Rx, Ry = Rx.cpu().numpy().astype(np.float64), Ry.cpu().numpy().astype(np.float64)
    for c in range(ncell):
        rx, ry = oracle.friction(p, h[:, c].astype(np.float64), Jx[:, c].astype(np.float64),
                                 Jy[:, c].astype(np.float64))
        scale = max(np.abs(rx).max(), np.abs(ry).max())
        assert np.abs(Rx[:, c] - rx).max() <= 1e-4 * scale + 1e-12
        assert np.abs(Ry[:, c] - ry).max() <= 1e-4 * scale + 1e-12


def test_full_size_film3_1024_in_bench_configuration():
    """The 1024 x 1024 three-layer workload in the launch configuration the
    benchmark times: three steps from a seeded non-equilibrium state, every
    population compared with the oracle."""
    p = workloads.film3_d2q9_params(1024, 1024)
    f = _f32(workloads.random_populations(7, p, 0.55, 1.05, 1e-3))
    hmax = oracle.heights(p, f).max()
    with B.Solver(p, oracle.heights(p, f)) as s:
        s.set_state(f)
        s.step(3)
        fg = s.get_state().astype(np.float64)
    fr = f
    for _ in range(3):
        fr = oracle.step(p, fr)
    assert np.abs(fg - fr).max() <= 3 * 4e-6 * hmax


def test_full_size_lens3_2048_in_bench_configuration():
    """The 2048 x 2048 three-layer lens field of the bench workloads (lenses
    of radius 200 on two flat layers, steep rims), in its launch
    configuration: three steps from the initial state, every population of
    the 12.6 M layer-sites compared with the oracle."""
    side, radius = 2048, 200.0
    p = workloads.lens3_params(side, side, radius)
    h0 = _f32(workloads.lens3_heights(side, side, radius))
    with B.Solver(p, h0) as s:
        s.step(3)
        fg = s.get_state().astype(np.float64)
        assert s.status() == B.MLSW_OK
    fr = oracle.run(p, oracle.init(p, h0.ravel()), 3)
    hmax = h0.max()
    assert np.abs(fg - fr).max() <= 3 * 4e-6 * hmax


def test_nonfinite_state_is_reported():
    p = workloads.film3_d2q9_params(40, 20)
    h0 = workloads.film3_d2q9_heights(40, 20)
    with B.Solver(p, h0) as s:
        f = s.get_state()
        f[1, 0, 7, 9] = np.nan
        s.set_state(f)
        s.step(1)
        assert s.status() == B.MLSW_ERR_NONFINITE
        assert s.status() == B.MLSW_OK  # cleared by the query
        h = np.array(h0, dtype=np.float32)
        h[2, 3, 3] = -0.5
        s.set_heights(h)
        with pytest.raises(B.MlswError) as e:
            s.get_heights()
        assert e.value.code == B.MLSW_ERR_NONFINITE


def test_checkpoint_resume_bit_exact():
    p = workloads.film3_d2q9_params(64, 48)
    h0 = workloads.film3_d2q9_heights(64, 48)
    with B.Solver(p, h0) as s, B.Solver(p, np.ones_like(h0)) as t:
        s.step(10)
        H, g = s.save_state()
        s.step(15)
        a = s.save_state()[1]
        t.load_state(H, g)  # a second handle resumes from the checkpoint
        t.step(15)
        assert np.array_equal(t.save_state()[1], a)
        assert np.array_equal(t.get_heights(), s.get_heights())


def test_state_get_set_roundtrip_is_exact_in_true_populations():
    p = workloads.film3_d2q9_params(40, 20)
    f = _f32(workloads.random_populations(23, p, 0.5, 1.0, 2e-3))
    with B.Solver(p, oracle.heights(p, f)) as s:
        s.set_state(f)
        # f_0 and H_i lie within a factor two of each other, so f_0 - H_i and
        # H_i + (f_0 - H_i) are exact in FP32
        assert np.array_equal(s.get_state().astype(np.float64), f)


def test_heights_roundtrip_and_diagnostics():
    p = workloads.film3_d2q9_params(48, 40)
    f = _f32(workloads.random_populations(17, p, 0.5, 1.0, 2e-3))
    h, Jx, Jy = oracle.moments(p, f)
    with B.Solver(p, h) as s:
        h32 = np.asarray(h, dtype=np.float32)
        assert np.array_equal(s.get_heights(), h32)
        s.set_state(f)
        mass, ke, hmin = s.get_diagnostics()
    np.testing.assert_allclose(mass, h.sum(axis=(1, 2)), rtol=1e-6)
    assert ke == pytest.approx(((Jx ** 2 + Jy ** 2) / (2 * h)).sum(), rel=1e-4)
    assert hmin == pytest.approx(h.min(), rel=1e-6)


def test_torch_stream_binding_and_launch_count():
    import torch
    p = workloads.film2_d1q3_params(512)
    h0 = workloads.film2_d1q3_heights(512)
    st = torch.cuda.Stream()
    with B.Solver(p, h0, stream=st) as a, B.Solver(p, h0) as b:
        a.step(40)
        b.step(40)
        assert np.array_equal(a.get_heights(), b.get_heights())
        # init (with ghost images), one persistent launch for the 40 steps of
        # this one-CTA D1Q3 lattice, read-out
        assert a.launch_count() == 1 + 1 + 1
    q = dict(p, flags=B.MLSW_FLAG_NO_PERSISTENT)
    with B.Solver(q, h0) as c:
        c.step(40)
        c.get_heights()
        assert c.launch_count() == 1 + 40 + 1


def test_pinned_host_heights_match_pageable():
    """Page-locked heights go through the kernels in place (no staging
    copy); the results equal those of pageable buffers bit for bit."""
    import torch
    p = workloads.film3_d2q9_params(72, 40)
    h0 = workloads.film3_d2q9_heights(72, 40).astype(np.float32)
    pin_in = torch.from_numpy(h0.copy()).pin_memory()
    pin_out = torch.zeros(h0.shape, dtype=torch.float32).pin_memory()
    with B.Solver(p, h0) as a, B.Solver(p, h0) as b:
        a.step(7)
        b.step(7)
        ref = a.get_heights()
        b.get_heights(pin_out.numpy())
        assert np.array_equal(pin_out.numpy(), ref)
        a.set_heights(h0)
        b.set_heights(pin_in.numpy())
        a.step(5)
        b.step(5)
        assert np.array_equal(a.get_state(), b.get_state())
        assert np.array_equal(a.get_heights(), b.get_heights(pin_out.numpy()))
        bad = h0.copy()
        bad[1, 3, 4] = -1.0
        pin_bad = torch.from_numpy(bad).pin_memory()
        with pytest.raises(B.MlswError):
            b.set_heights(pin_bad.numpy())
            b.get_heights(pin_out.numpy())


def test_set_heights_from_device_memory_equals_host():
    """mlswlbm_set_heights_device restarts the state exactly as the host
    call does, and bad heights set the status."""
    import torch
    p = workloads.random_params(77, 3, B.MLSW_D2Q9, 72, 40)
    h0 = workloads.random_heights(78, p).astype(np.float32)
    with B.Solver(p, h0) as a, B.Solver(p, h0) as b:
        a.step(9)
        b.step(9)
        h1 = workloads.random_heights(79, p).astype(np.float32)
        a.set_heights(h1)
        b.set_heights_device(torch.from_numpy(h1).cuda())
        torch.cuda.synchronize()
        assert np.array_equal(a.get_state(), b.get_state())
        a.step(4)
        b.step(4)
        assert np.array_equal(a.get_heights(), b.get_heights())
        bad = h1.copy()
        bad[0, 1, 2] = 0.0
        b.set_heights_device(torch.from_numpy(bad).cuda())
        assert b.status() == B.MLSW_ERR_NONFINITE


@pytest.mark.parametrize("n,nx,ny", [(3, 1024, 1024), (1, 1024, 1024), (5, 512, 400)])
def test_large_pinned_read_out_matches_pageable(n, nx, ny):
    """Large page-locked outputs (up to 12.6 MB, one to five layers) are
    written in place by the read-out kernel: same bits as the pageable
    path, again after further steps."""
    import torch
    p = workloads.random_params(60 + n, n, B.MLSW_D2Q9, nx, ny)
    h0 = workloads.random_heights(70 + n, p).astype(np.float32)
    pin_out = torch.zeros(h0.shape, dtype=torch.float32).pin_memory()
    with B.Solver(p, h0) as a:
        a.step(3)
        ref = a.get_heights()
        out = a.get_heights(pin_out.numpy())
        assert out is pin_out.numpy() or np.shares_memory(out, pin_out.numpy())
        assert np.array_equal(pin_out.numpy(), ref)
        a.step(2)
        ref2 = a.get_heights()
        a.get_heights(pin_out.numpy())
        assert np.array_equal(pin_out.numpy(), ref2)
        assert a.status() == B.MLSW_OK


PERSIST = [(1, 1.0, 512, 3), (2, 1.0, 512, 3), (3, 0.8, 37, 2), (4, 1.0, 1, 3), (5, 1.3, 2, 3),
           (2, 1.0, 3, 2), (3, 1.0, 1000, 3)]


@pytest.mark.parametrize("n,tau,nx,nw", PERSIST)
def test_d1q3_persistent_matches_per_step_launches_bit_exact(n, tau, nx, nw):
    """The one-CTA persistent D1Q3 kernel runs the same cell arithmetic as
    the per-step kernel: states agree bit for bit, tiny and odd sizes
    included, for tau = 1 and tau != 1."""
    p = workloads.random_params(100 + n, n, B.MLSW_D1Q3, nx, 1, tau=tau)
    p["nw"], p["mw"] = (3, 2) if nw == 3 else (4, 2)
    h0 = workloads.random_heights(200 + n, p)
    q = dict(p, flags=B.MLSW_FLAG_NO_PERSISTENT)
    with B.Solver(p, h0) as a, B.Solver(q, h0) as b:
        a.step(25)
        b.step(25)
        assert np.array_equal(a.get_state(), b.get_state())
        a.step(1)
        b.step(1)
        assert np.array_equal(a.get_heights(), b.get_heights())
        assert a.status() == B.MLSW_OK


def test_d1q3_persistent_chunked_long_run():
    """More steps than one persistent launch takes (16384): the chunks hand
    the state over exactly."""
    p = workloads.film2_d1q3_params(512)
    h0 = workloads.film2_d1q3_heights(512)
    q = dict(p, flags=B.MLSW_FLAG_NO_PERSISTENT)
    with B.Solver(p, h0) as a, B.Solver(q, h0) as b:
        a.step(16384 + 7)
        b.step(16384 + 7)
        assert np.array_equal(a.get_state(), b.get_state())


# --------------------------------------------------------------------------
# droplet and lens equilibria: the GPU is compared with the oracle by the
# fitted angles (section "Droplet equilibria"), not cell by cell. Over
# 1e4-2e4 steps the FP32 heights drift from the FP64 ones by a few 1e-5
# of the drop height, which moves a fitted angle by a few 0.01 degrees and
# E by a few 1e-3: the bounds are 0.1 degree and 0.005, a tenth of the
# paper's own fit accuracy (E < 2-5 %)
# --------------------------------------------------------------------------
def _gpu_relaxed(p, h0, steps):
    with B.Solver(p, h0) as s:
        s.step(steps)
        h = s.get_heights().astype(np.float64)
        assert s.status() == B.MLSW_OK
    return h


def _oracle_relaxed(p, h0, steps):
    f = oracle.run(p, oracle.init(p, _f32(h0).ravel()), steps)
    return oracle.heights(p, f).reshape(np.shape(h0))


def test_sessile_ridge_angle_matches_oracle():
    p = workloads.drop1d_params(128, 20.0)
    h0 = workloads.drop1d_heights(128, 20.0)
    tg, eg = droplets.fit_angle_1d(_gpu_relaxed(p, h0, 20000), p["hstar"])
    to, eo = droplets.fit_angle_1d(_oracle_relaxed(p, h0, 20000), p["hstar"])
    assert abs(tg - to) < 0.1 and abs(eg - eo) < 0.005
    assert abs(tg - 20.0) < 1.5


def test_lens_angles_match_oracle():
    p = workloads.lens1d_params(160, 20.0)
    h0 = workloads.lens1d_heights(160, 20.0)
    g = droplets.lens_angles_1d(_gpu_relaxed(p, h0, 20000), p["hstar"])
    o = droplets.lens_angles_1d(_oracle_relaxed(p, h0, 20000), p["hstar"])
    for (tg, eg), (to, eo) in zip(g, o):
        assert abs(tg - to) < 0.1 and abs(eg - eo) < 0.005
        assert abs(tg - 20.0) < 1.5


def test_three_layer_lens_field_128_matches_oracle_angles():
    """The 128 x 128 version of the 2048 x 2048 lens workload: after 10000
    steps every lens's opening angles agree with the oracle's (stored by
    tests/golden/make_lens3_128.py) and lie near Neumann's 20 degrees."""
    with open(os.path.join(os.path.dirname(__file__), "golden", "lens3_128_angles.json")) as fh:
        gold = json.load(fh)
    p = workloads.lens3_params(128, 128, 12.5)
    h0 = workloads.lens3_heights(128, 128, 12.5)
    h = _gpu_relaxed(p, h0, gold["steps"])
    ang = droplets.lens3_angles(h, workloads.lens3_centres(128, 128, 12.5), 12.5)
    for (up, lo), gu, gl in zip(ang, gold["upper"], gold["lower"]):
        assert abs(up[0] - gu[0]) < 0.1 and abs(lo[0] - gl[0]) < 0.1
        assert abs(up[0] - 20.0) < 2.0 and abs(lo[0] - 20.0) < 2.0
        assert up[1] < 0.05 and lo[1] < 0.05
    # per-layer mass after 1e4 FP32 steps, the precursor-dominated lens layer
    # included: the collision hands the rounding error of the shifted rest
    # population on to two moving populations, so mass is kept to FP32
    # round-off (V5), against the FP64 oracle's (conserved to 1e-13)
    np.testing.assert_allclose(h.sum(axis=(1, 2)), gold["mass"], rtol=1e-6)


# --------------------------------------------------------------------------
# free energy (Eq. free_energy_n_layer) and the kinetic-energy stop
# criterion of equilibrium runs
# --------------------------------------------------------------------------
@pytest.mark.parametrize("lat", [1, 2])
def test_free_energy_matches_the_formula_on_read_back_heights(lat):
    if lat == 2:
        p = workloads.random_params(41, 3, B.MLSW_D2Q9, 72, 40, multilayer_S=True)
    else:
        p = workloads.random_params(42, 4, B.MLSW_D1Q3, 300, 1, multilayer_S=True)
    with B.Solver(p, workloads.random_heights(43, p)) as s:
        s.step(50)
        F = s.free_energy()
        want = droplets.free_energy(p, s.get_heights().astype(np.float64))
    assert F == pytest.approx(want, rel=1e-10, abs=1e-12)


def test_free_energy_decreases_while_a_film_dewets():
    g, th = 0.01, np.radians(30)
    S = g * (np.cos(th) - 1)
    p = dict(n=2, lattice=1, nx=128, ny=1, tau=1.0, gamma=[g, g], S=[[S, 0.0], [S]],
             mu=[1 / 6, 1 / 6], beta=[1.0, 1.0], nw=3, mw=2, hstar=0.05)
    rng = np.random.default_rng(7)
    h0 = (0.25 + 1e-3 * rng.uniform(-1, 1, (2, 1, 128)))
    with B.Solver(p, h0) as s:
        F = []
        for _ in range(25):
            F.append(s.free_energy())
            s.step(1000)
        hmin = s.get_heights().min()
    assert np.all(np.diff(F) <= 1e-9 * abs(F[0]))
    assert F[-1] < 0.97 * F[0] and hmin < 0.06


def test_step_until_stops_on_kinetic_energy():
    p = workloads.lens3_params(128, 128, 12.5)
    h0 = workloads.lens3_heights(128, 128, 12.5)
    with B.Solver(p, h0) as s:
        done, ke = s.step_until(200000, 500, 2e-6)
        assert ke < 2e-6 and 0 < done < 200000 and done % 500 == 0
        _, ke2, _ = s.get_diagnostics()
        assert ke2 == ke
        # a threshold met at the first check: one chunk is taken
        done2, _ = s.step_until(1000, 100, 1.0)
        assert done2 == 100
        # a threshold out of reach: stops at max_steps
        done3, ke3 = s.step_until(700, 300, 0.0)
        assert done3 == 700 and ke3 > 0.0


# --------------------------------------------------------------------------
# corrugated substrate z_0 = A cos(2 pi (kx x / nx + ky y / ny))
# --------------------------------------------------------------------------
SUB_ONE_STEP = [(n, lat, tau) for n in (1, 2, 3, 5) for lat, tau in ((2, 1.0), (2, 0.8), (1, 1.0))]


@pytest.mark.parametrize("n,lat,tau", SUB_ONE_STEP)
def test_one_step_on_a_corrugated_substrate(n, lat, tau):
    p, f = one_step_case(n, lat, tau)
    p = dict(p, sub_amp=0.2, sub_kx=3, sub_ky=0 if lat == 1 else 2)
    hmax = oracle.heights(p, f).max()
    with B.Solver(p, oracle.heights(p, f)) as s:
        s.set_state(f)
        s.step(1)
        fg = s.get_state().astype(np.float64)
        assert s.status() == B.MLSW_OK
    fr = oracle.step(p, f)
    assert np.abs(fg - fr).max() <= 4e-6 * hmax


@pytest.mark.parametrize("lat", [1, 2])
def test_film_on_a_corrugated_substrate_multistep(lat):
    if lat == 2:
        p = dict(workloads.random_params(61, 2, 2, 45, 33), sub_amp=0.05, sub_kx=2, sub_ky=1)
        steps = 300
    else:  # the persistent one-CTA kernel
        p = dict(workloads.random_params(62, 2, 1, 128, 1), sub_amp=0.05, sub_kx=3, sub_ky=0)
        steps = 1000
    h0 = workloads.random_heights(63, p, 0.5, 1.1, 2e-3)
    hg, hr = _run_both(p, h0, steps)
    assert _relmax(hg, hr) <= 1e-5


def test_substrate_translation_by_one_period_is_bit_exact():
    # z_0 with kx = 4 on 64 columns and ky = 2 on 40 rows repeats after 16
    # columns and 20 rows; shifting the film by that moves every cell to a
    # new tile position over the same substrate height
    p = dict(workloads.random_params(64, 3, 2, 64, 40), sub_amp=0.1, sub_kx=4, sub_ky=2)
    h0 = workloads.random_heights(65, p, 0.5, 1.1, 1e-2).astype(np.float32)
    hs = np.roll(np.roll(h0, 16, axis=2), 20, axis=1)
    with B.Solver(p, h0) as a, B.Solver(p, hs) as b:
        a.step(40)
        b.step(40)
        ha, hb = a.get_heights(), b.get_heights()
    assert np.array_equal(np.roll(np.roll(ha, 16, axis=2), 20, axis=1), hb)


@pytest.mark.parametrize("lat", [1, 2])
def test_free_energy_on_a_corrugated_substrate(lat):
    if lat == 2:
        p = dict(workloads.random_params(66, 2, 2, 40, 24), sub_amp=0.1, sub_kx=1, sub_ky=2)
    else:
        p = dict(workloads.random_params(67, 3, 1, 200, 1), sub_amp=0.1, sub_kx=2, sub_ky=0)
    with B.Solver(p, workloads.random_heights(68, p)) as s:
        s.step(30)
        F = s.free_energy()
        want = droplets.free_energy(p, s.get_heights().astype(np.float64))
    assert F == pytest.approx(want, rel=1e-10, abs=1e-12)


# --------------------------------------------------------------------------
# a long dewetting run against the oracle by statistics: after rupture the
# FP32 and FP64 runs part cell by cell, so what is compared is the rupture
# step, the spectra before it and the distribution of heights after it
# (stored by tests/golden/make_dewet2_64.py)
# --------------------------------------------------------------------------
def test_long_dewetting_run_matches_oracle_statistics():
    with open(os.path.join(os.path.dirname(__file__), "golden", "dewet2_64_stats.json")) as fh:
        gold = json.load(fh)
    p = workloads.dewet2_params(64)
    h0 = workloads.dewet2_heights(64)
    with B.Solver(p, h0) as s:
        state = {"t": 0}

        def at(t):
            s.step(t - state["t"])
            state["t"] = t
            return s.get_heights().astype(np.float64)

        tr, _ = droplets.rupture_step(at, p["hstar"], gold["every"], 20000)
    assert abs(tr - gold["rupture_step"]) <= 0.03 * gold["rupture_step"]
    with B.Solver(p, h0) as s:
        m0, _, _ = s.get_diagnostics()
        s.step(gold["spectrum_step"])
        h_pre = s.get_heights().astype(np.float64)
        s.step(gold["post_step"] - gold["spectrum_step"])
        h_post = s.get_heights().astype(np.float64)
        m1, _, _ = s.get_diagnostics()
        assert s.status() == B.MLSW_OK
    for i in range(2):
        got = droplets.radial_spectrum(h_pre[i])
        want = np.array(gold["spectra"][i])
        assert np.linalg.norm(got - want) <= 0.05 * np.linalg.norm(want)
    # per-layer mass after ~2e4 FP32 steps, with half of each layer on its
    # precursor, far from the rest-population shift fixed at create: kept to
    # FP32 round-off (V5, 1e-6), against the run's own start and against the
    # FP64 oracle. Rounding the shifted rest population alone, without
    # handing its error on, drifted 4.5e-5 here.
    np.testing.assert_allclose(m1, m0, rtol=1e-6)
    np.testing.assert_allclose(h_post.sum(axis=(1, 2)), gold["mass"], rtol=1e-6)
    frac = (h_post[1] < 2 * p["hstar"]).mean()
    assert abs(frac - gold["dewetted_fraction"]) <= 0.03
    hist, _ = np.histogram(h_post[1], bins=np.array(gold["hist_bins"]))
    assert np.abs(hist / hist.sum() - np.array(gold["hist_upper"])).sum() <= 0.15


def test_bounded_wait_reports_timeout_and_the_context_survives():
    # the step kernels wait for their tile copies on an mbarrier with an
    # iteration limit; here a barrier that never gets its arrival makes the
    # same wait run out: the kernel records the timeout and returns
    assert B.selftest_bounded_wait(True, 256) == B.MLSW_OK
    assert B.selftest_bounded_wait(False, 256) == B.MLSW_ERR_TIMEOUT
    assert B.selftest_bounded_wait(False, 4096) == B.MLSW_ERR_TIMEOUT
    # and the CUDA context is fine afterwards
    p = workloads.film3_d2q9_params(40, 24)
    h0 = workloads.film3_d2q9_heights(40, 24)
    with B.Solver(p, h0) as s:
        s.step(5)
        assert s.status() == B.MLSW_OK
    assert B.selftest_bounded_wait(True, 256) == B.MLSW_OK


# --------------------------------------------------------------------------
# power spectra on the device (mlswlbm_get_spectrum) against the FFT of the
# read-back heights (tests/droplets.radial_spectrum, pinned on the CPU).
# The device transforms h - H_i in FP32 (log2 N radix-2 stages, each adding
# a few u of the transformed signal); the reference transforms, in FP64, the
# heights as read back, rounded to FP32 (error e <= u |h| / 2 per cell). That
# rounding moves |H(k)|^2 by at most 2 |H(k)| sqrt(N) e for N cells (the DFT
# of the rounding field has norm sqrt(N) e per mode on average; 3 sigma), so
# a bin with power P agrees to 1e-4 P + 6 sqrt(N P) e; bins below 1e-8 of
# the largest are only bounded.
# --------------------------------------------------------------------------
def _check_spectrum(s, h, nbins):
    got = s.spectrum(nbins)
    for i in range(h.shape[0]):
        f = h[i] if h.ndim == 3 else h[i][None, :]
        want = droplets.radial_spectrum(f, nbins)
        e = np.finfo(np.float32).eps * np.abs(f).max() / 2
        tol = 1e-4 * want + 6 * np.sqrt(f.size * want) * e
        big = want > 1e-8 * want.max()
        assert np.all(np.abs(got[i] - want)[big] <= tol[big]), i
        assert np.all(np.abs(got[i] - want)[~big] <= 1e-6 * want.max()), i


@pytest.mark.parametrize("nx,ny", [(128, 128), (256, 64), (64, 512)])
def test_spectrum_matches_fft_of_read_back_heights(nx, ny):
    p = workloads.film3_d2q9_params(nx, ny)
    h0 = workloads.film3_d2q9_heights(nx, ny, seed=4)
    with B.Solver(p, h0) as s:
        s.step(300)
        h = s.get_heights().astype(np.float64)
        _check_spectrum(s, h, min(nx, ny) // 2)
        _check_spectrum(s, h, 7)


def test_spectrum_d1q3_and_a_single_mode():
    p = workloads.film2_d1q3_params(512)
    h0 = workloads.film2_d1q3_heights(512)
    with B.Solver(p, h0) as s:
        s.step(200)
        _check_spectrum(s, s.get_heights().astype(np.float64), 256)
    # one cosine mode (3, 4) of amplitude a on layer 2 only: all its power
    # sits in bin 5, |H(k)|^2 = (a N / 2)^2 at k = +-(3, 4)
    nx = ny = 64
    p = workloads.film3_d2q9_params(nx, ny)
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    a = 1e-3
    h = np.stack([np.full((ny, nx), 1.0), 0.8 + a * np.cos(2 * np.pi * (3 * x / nx + 4 * y / ny)),
                  np.full((ny, nx), 0.6)])
    with B.Solver(p, h) as s:
        sp = s.spectrum(32)
        counts = np.bincount(np.rint(np.hypot(*np.meshgrid(np.fft.fftfreq(nx) * nx,
                                                           np.fft.fftfreq(ny) * ny))).astype(int).ravel())
        want5 = 2 * (a * nx * ny / 2) ** 2 / counts[5]
        assert abs(sp[1, 5] - want5) <= 1e-4 * want5
        others = np.delete(sp[1], 5)
        assert others.max() <= 1e-8 * want5
        assert sp[0].max() <= 1e-8 * want5 and sp[2].max() <= 1e-8 * want5


def test_spectrum_rejects_unsupported_sizes():
    p = workloads.film3_d2q9_params(96, 64)
    with B.Solver(p, workloads.film3_d2q9_heights(96, 64)) as s:
        with pytest.raises(B.MlswError) as err:
            s.spectrum(16)
        assert err.value.code == B.MLSW_ERR_UNSUPPORTED
        assert s.status() == B.MLSW_OK


def test_spectrum_growth_follows_the_linearised_step():
    """The spinodal-dewetting analysis of the paper on the device: a film
    seeded with small white noise in every layer, stepped t times, has the
    radial spectrum that the independently linearised step (tests/lsa.py)
    predicts when G(k)^t is applied to every Fourier mode of the initial
    heights, bin by bin. At noise 1e-4 the FP32 step and the neglected
    second-order terms move a mode by ~2e-3 of its amplitude over t steps
    (the single-mode batch check), so the bins agree to 1 % of their power;
    bins whose modes have decayed below 1e-4 of the largest bin are only
    bounded."""
    # the spinodal three-layer film of the bench (modes 1-2 grow, the rest
    # decay at rates spread over three decades)
    side, n, t, eps = 64, 3, 2000, 1e-4
    p = workloads.film3_d2q9_params(side, side)
    h0 = np.array([1.0, 0.8, 0.6])
    rng = np.random.default_rng(31)
    h = (h0[:, None, None] + eps * rng.standard_normal((n, side, side))).astype(np.float32)
    with B.Solver(p, h) as s:
        s.step(t)
        got = s.spectrum(side // 2)
        assert s.status() == B.MLSW_OK
    H0 = np.fft.fft2(h.astype(np.float64), axes=(1, 2))
    k1 = np.fft.fftfreq(side) * side
    KX, KY = np.meshgrid(k1, k1)  # [ky][kx]
    Q = 9
    Ht = np.zeros_like(H0)
    for iy in range(side):
        for ix in range(side):
            if ix == 0 and iy == 0:
                continue
            G = lsa.step_matrix(p, h0, (2 * np.pi * KX[iy, ix] / side, 2 * np.pi * KY[iy, ix] / side))
            v = np.zeros(n * Q, dtype=complex)
            v[0::Q] = H0[:, iy, ix]
            Ht[:, iy, ix] = (np.linalg.matrix_power(G, t) @ v).reshape(n, Q).sum(axis=1)
    b = np.rint(np.hypot(KX, KY)).astype(int).ravel()
    nb = side // 2
    keep = b < nb
    cnt = np.bincount(b[keep], minlength=nb)
    for i in range(n):
        P = (np.abs(Ht[i]) ** 2).ravel()
        want = np.bincount(b[keep], weights=P[keep], minlength=nb) / np.maximum(cnt, 1)
        big = want > 1e-4 * want.max()
        assert np.all(np.abs(got[i] - want)[big] <= 1e-2 * want[big]), (i, got[i][big] / want[big])
        assert np.all(np.abs(got[i] - want)[~big] <= 1e-4 * want.max()), i


def test_radial_profiles_on_the_device_and_the_library_cap_fit():
    """mlswlbm_get_radial_profile equals the azimuthal means of the read-back
    interfaces (tests/droplets.radial_profile) ring by ring, substrate
    included, and the library's arc fit on those profiles gives the lens
    angles of the host helper that the oracle comparison uses."""
    side, radius = 128, 12.5
    p = workloads.lens3_params(side, side, radius)
    h0 = workloads.lens3_heights(side, side, radius)
    for sub in (False, True):
        q = dict(p, sub_amp=0.05, sub_kx=1, sub_ky=2) if sub else p
        with B.Solver(q, h0) as s:
            s.step(3000)
            h = s.get_heights().astype(np.float64)
            y, x = np.meshgrid(np.arange(side), np.arange(side), indexing="ij")
            z0 = 0.05 * np.cos(2 * np.pi * (x / side + 2 * y / side)) if sub else np.zeros_like(h[0])
            z = np.concatenate([z0[None], z0[None] + np.cumsum(h, axis=0)])
            nb = int(1.6 * radius)
            for c in workloads.lens3_centres(side, side, radius):
                cc = droplets.peak_centre(h[2], c, int(radius))
                prof, cnt = s.radial_profile(cc, nb)
                for m in range(4):
                    rad, want, area = droplets.radial_profile(z[m], cc, nb)
                    assert np.array_equal(cnt, area.astype(np.int64))
                    np.testing.assert_allclose(prof[m], want, rtol=1e-12, atol=1e-13)
                if sub:
                    continue
                # upper and lower opening angles, as tests/droplets.lens3_angles forms them
                (up_ref, lo_ref), = droplets.lens3_angles(h, [c], radius)
                up = prof[3] - prof[3][-3:].mean()
                lo = prof[2][-3:].mean() - prof[2]
                t_up, e_up = B.fit_cap_angle(up, cnt, 0.0)
                t_lo, e_lo = B.fit_cap_angle(lo, cnt, 0.0)
                assert abs(t_up - up_ref[0]) < 1e-6 and abs(e_up - up_ref[1]) < 1e-9
                assert abs(t_lo - lo_ref[0]) < 1e-6 and abs(e_lo - lo_ref[1]) < 1e-9
            assert s.status() == B.MLSW_OK


def test_analysis_edge_cases():
    """More bins than wavevectors or cells reach (empty bins are 0), a
    centre outside the box (periodic distances), one-row and tiny lattices,
    and argument errors that leave the handle usable."""
    p = workloads.film3_d2q9_params(32, 16)
    h0 = workloads.film3_d2q9_heights(32, 16, seed=3)
    with B.Solver(p, h0) as s:
        s.step(20)
        h = s.get_heights().astype(np.float64)
        sp = s.spectrum(64)  # |k| reaches round(sqrt(16^2 + 8^2)) = 18
        for i in range(3):
            want = droplets.radial_spectrum(h[i], 64)
            np.testing.assert_allclose(sp[i, :19], want[:19], rtol=1e-3, atol=1e-6 * want.max())
            assert np.all(sp[i, 19:] == 0)
        z = np.concatenate([np.zeros((1, 16, 32)), np.cumsum(h, axis=0)])
        for c in [(-3.5, 40.25), (31.0, 15.0), (100.0, -20.0)]:
            prof, cnt = s.radial_profile(c, 40)
            for m in range(4):
                _, want, area = droplets.radial_profile(z[m], np.mod(c, (32, 16)), 40)
                np.testing.assert_allclose(prof[m], want, rtol=1e-12, atol=1e-13)
            assert cnt.sum() == 32 * 16 and np.all(cnt[20:] == 0)
        with pytest.raises(B.MlswError) as err:
            s.radial_profile((0.0, 0.0), 0)
        assert err.value.code == B.MLSW_ERR_ARG
        with pytest.raises(B.MlswError) as err:
            s.spectrum(0)
        assert err.value.code == B.MLSW_ERR_ARG
        assert s.status() == B.MLSW_OK
    # D1Q3: spectra yes, ring profiles no
    p = workloads.film2_d1q3_params(64)
    with B.Solver(p, workloads.film2_d1q3_heights(64)) as s:
        assert s.spectrum(32).shape == (2, 32)
        with pytest.raises(B.MlswError) as err:
            s.radial_profile((10.0, 0.0), 8)
        assert err.value.code == B.MLSW_ERR_UNSUPPORTED
