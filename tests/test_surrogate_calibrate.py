"""CPU checks of surrogate.calibrate: the largest threshold on the predicted
change under which the wanted fraction of windows meets the error bound."""
import numpy as np

from paper_2409_16659_gb300 import surrogate as S


def test_calibrate_on_a_hand_made_table():
    change = np.array([[1e-4, 2e-4, 3e-4, 4e-4, 5e-4]])
    err = np.array([[5e-4, 8e-4, 2e-3, 9e-4, 4e-3]])
    # every window up to change 2e-4 is within 1e-3; the third is not
    assert S.calibrate(err, change) == 2e-4
    # in order of change the running fraction within the bound is 1, 1, 2/3, 3/4, 3/5
    assert S.calibrate(err, change, quantile=0.75) == 4e-4
    assert S.calibrate(err, change, quantile=0.6) == 5e-4


def test_calibrate_with_no_qualifying_window_returns_zero():
    change = np.array([[1e-4, 2e-4]])
    err = np.array([[5e-3, 1e-3 + 1e-9]])
    assert S.calibrate(err, change) == 0.0


def test_calibrate_ignores_the_order_of_the_table():
    rng = np.random.default_rng(3)
    change = rng.uniform(0, 1e-3, (4, 30))
    err = change * rng.uniform(0.5, 3.0, change.shape)
    perm = rng.permutation(change.size)
    a = S.calibrate(err, change, quantile=0.9)
    b = S.calibrate(err.ravel()[perm], change.ravel()[perm], quantile=0.9)
    assert a == b
    # the threshold's windows meet the bound in at least 90 % of cases
    sel = change.ravel() <= a
    assert (err.ravel()[sel] <= 1e-3).mean() >= 0.9
