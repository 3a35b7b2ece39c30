"""The contact-angle fit of the C library (mlswlbm_fit_cap_angle, host
code, no GPU): it recovers the angle of a circular cap, equals the test
helper that fits the oracle's and the GPU's drops (tests/droplets.py: same
objective E(theta), scan and refinement, written independently), and
rejects bad arguments."""
import math

import numpy as np
import pytest

import workloads
from paper_2409_16659_gb300 import mlswlbm as B
from tests import droplets


def _helper(prof, area, base):
    rad = np.arange(prof.size) + 0.5
    t, e = droplets._scan_min(lambda th: droplets._radial_err(rad, prof, area, base, th))
    return math.degrees(t), e


@pytest.mark.parametrize("theta,base", [(12.0, 0.1), (23.0, 0.2), (41.0, 0.0)])
def test_fit_recovers_a_cap(theta, base):
    rad = np.arange(40) + 0.5
    area = 2 * np.pi * rad
    # a cap whose apex is at r = 0; the rings sample it at r = b + 1/2
    rc = 20.0
    peak = base + rc * (1 - math.cos(math.radians(theta)))
    prof = workloads.cap_profile(rad, peak, base, math.radians(theta))
    t, e = B.fit_cap_angle(prof, area, base)
    th, eh = _helper(prof, area, base)
    assert abs(t - th) < 1e-7 and abs(e - eh) < 1e-10
    # the first ring sits half a cell below the apex: the fit lands within
    # a quarter degree of the true angle, with E well under 1 %
    assert abs(t - theta) < 0.25 and e < 1e-2


def test_fit_matches_the_helper_on_a_perturbed_profile():
    rng = np.random.default_rng(5)
    rad = np.arange(25) + 0.5
    area = np.rint(2 * np.pi * rad)
    prof = workloads.cap_profile(rad, 2.5, 0.15, math.radians(17.0)) + 2e-3 * rng.standard_normal(25)
    prof[0] = max(prof[0], 2.5)
    t, e = B.fit_cap_angle(prof, area, 0.15)
    th, eh = _helper(prof, area, 0.15)
    assert abs(t - th) < 1e-7 and abs(e - eh) < 1e-10


def test_fit_rejects_bad_arguments():
    with pytest.raises(B.MlswError):
        B.fit_cap_angle([0.1, 0.2, 0.3], [1, 1, 1], 0.5)   # apex below the base
    with pytest.raises(B.MlswError):
        B.fit_cap_angle([1.0], [1.0], 0.0)                  # one ring
    with pytest.raises(ValueError):
        B.fit_cap_angle([1.0, 0.5], [1.0], 0.0)


def test_radial_profile_reference_exact_cases():
    """The ring means that the device profiles are checked against: a
    constant field is that constant in every ring, a field equal to floor(r)
    around the centre (periodic distances) is b in ring b, and every cell
    lies in exactly one ring."""
    ny, nx = 24, 40
    centre = (13.25, 7.5)
    y, x = np.meshgrid(np.arange(ny, dtype=float), np.arange(nx, dtype=float), indexing="ij")
    dx = x - centre[0]
    dx -= nx * np.round(dx / nx)
    dy = y - centre[1]
    dy -= ny * np.round(dy / ny)
    r = np.hypot(dx, dy)
    nb = int(r.max()) + 1
    rad, prof, area = droplets.radial_profile(np.full((ny, nx), 2.5), centre, nb)
    assert np.all(prof[area > 0] == 2.5) and area.sum() == nx * ny
    rad, prof, area = droplets.radial_profile(np.floor(r), centre, nb)
    nz = area > 0
    np.testing.assert_array_equal(prof[nz], np.arange(nb)[nz])
    np.testing.assert_array_equal(rad, np.arange(nb) + 0.5)
