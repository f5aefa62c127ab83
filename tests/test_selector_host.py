"""Host-side logic of the grid selector: the check's calibration (no GPU needed)."""
import math

import numpy as np

from paper_1612_01799_gb300 import selector as S


def test_calibration_is_monotone_and_conservative():
    rng = np.random.default_rng(0)
    # error ~ eta above a round-off floor of 1e-7, with scatter; eta keeps falling below it
    leta = rng.uniform(-9.0, 0.0, 5000)
    lerr = np.maximum(leta + 0.5 + 0.2 * rng.standard_normal(leta.size), -7.0 + 0.05 * rng.standard_normal(leta.size))
    cal = S.calibrate(leta, lerr, quantile=0.98)
    b = np.array(cal["bound"])
    assert np.all(np.diff(b) >= 0)
    # about 2% of the pairs above their bin's bound (interpolated quantiles in finite bins)
    above = [lerr[i] > S.calibrated_bound(cal, 10.0 ** leta[i]) for i in range(leta.size)]
    assert np.mean(above) <= 0.03
    # the floor does not flatten the map: tol 1e-6 is accepted for small eta, not for large
    assert S.calibrated_bound(cal, 1e-8) <= -6.0
    assert S.calibrated_bound(cal, 1e-3) > -6.0
    thr = S.eta_threshold(cal, 1e-6)
    assert 1e-8 < thr < 1e-5
    assert S.calibrated_bound(cal, thr * 0.999) <= -6.0
    # beyond the training range the check refuses
    assert S.calibrated_bound(cal, 10.0) == math.inf


def test_calibration_small_bins_use_their_maximum():
    cal = S.calibrate(np.array([-3.0, -3.1, -1.0]), np.array([-5.0, -4.0, -2.0]), width=0.5, min_count=4)
    assert S.calibrated_bound(cal, 10 ** -3.05) == -4.0
    assert S.calibrated_bound(cal, 10 ** -1.0) == -2.0
    assert S.calibrated_bound(cal, 10 ** -2.0) == -4.0        # empty bin keeps the running maximum
