"""Host-side rules of the learned start (paper_2104_07146_gb300/learned_start.py)
on the CPU, with the perceptron's output supplied directly: the prediction
becomes a theta through the Sec. 5 transform, the simplex steps are the
exponentiated log scales clipped to [0.05, 2], and a prediction that is not
finite or lands outside the admissible range falls back to the default start
with unit steps.  Also the prior box of the simulated training fields."""
import math

import numpy as np
import pytest

import oracle
from paper_2104_07146_gb300 import learned_start as ls


class _Fixed(ls.LearnedStart):
    # the rules of start() around a given network output (no device)
    def __init__(self, y):
        self._y = np.asarray(y, dtype=np.float32).reshape(1, 8)

    def forward(self, feats):
        return self._y

    def close(self):
        pass


def _start(y, monkeypatch):
    monkeypatch.setattr(ls, "features", lambda ctx, locs, Z: np.zeros(ls.NF, dtype=np.float32))
    m = _Fixed(y)
    m.ctx = None
    return m.start(None, None)


def test_prediction_maps_through_the_transform(monkeypatch):
    x = oracle.untransform((0.12, 0.9, 1.4, 0.02))
    th, steps, fb = _start(list(x) + [math.log(0.5), math.log(3.0), math.log(0.01), 0.0],
                           monkeypatch)
    assert not fb
    np.testing.assert_allclose(th, (0.12, 0.9, 1.4, 0.02), rtol=1e-5)   # FP32 output
    np.testing.assert_allclose(steps, [0.5, 2.0, 0.05, 1.0], rtol=1e-6)


@pytest.mark.parametrize("y", [
    [math.nan, 0, 0, 0, 0, 0, 0, 0],                 # not finite
    [0, 0, 0, 0, math.inf, 0, 0, 0],
    [0, -40.0, 0, 0, 0, 0, 0, 0],                    # ell = 1.5^40: above 1e3
    [0, 0, -25.0, 0, 0, 0, 0, 0],                    # nu = 1.2^25 = 95: above 20
])
def test_fallback_to_the_default_start(y, monkeypatch):
    th, steps, fb = _start(y, monkeypatch)
    assert fb and th == ls.DEFAULT_THETA0 and steps == [1.0, 1.0, 1.0, 1.0]


def test_training_thetas_stay_in_the_prior_box():
    lo = {k: v[0] for k, v in ls.PRIOR.items()}
    hi = {k: v[1] for k, v in ls.PRIOR.items()}
    th = np.array([ls.draw_theta(11, i) for i in range(400)])
    for j, k in enumerate(("ell", "nu", "sigma2", "tau2")):
        assert np.all(th[:, j] >= lo[k]) and np.all(th[:, j] <= hi[k])
    # ell, sigma2, tau2 log-uniform, nu uniform: medians near the centres
    for j, k in ((0, "ell"), (2, "sigma2"), (3, "tau2")):
        assert abs(np.log(np.median(th[:, j])) - 0.5 * (np.log(lo[k]) + np.log(hi[k]))) < 0.35
    assert abs(np.median(th[:, 1]) - 0.5 * (lo["nu"] + hi["nu"])) < 0.15
