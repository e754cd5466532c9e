"""The optimiser of hmle_fit (Nelder-Mead, host code of the library) against
the oracle's Nelder-Mead, on the CPU.

hmle_nelder_mead runs the same template as hmle_fit / hmle_fit_profiled on a
caller's objective.  Both implementations follow the same rules
(reflection 1, expansion 2, contraction 1/2, shrink 1/2, stable ordering,
f- and x-spread stopping rule), so on these objectives they take the same
path: the same iterations and evaluation counts and the same best vertex up
to the rounding of the centroid.  The tolerances stop each run before the
simplex shrinks to where f differs only by rounding: there the two
implementations' last-bit differences in the centroid decide comparisons
and the paths may part.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2104_07146_gb300 import hmle


def rosenbrock(x):
    return float(np.sum(100.0 * (x[1:] - x[:-1] ** 2) ** 2 + (1.0 - x[:-1]) ** 2))


def weighted_quadratic(x):
    return float(np.sum((np.arange(1, x.size + 1) * (x - 0.3)) ** 2))


def boxed(x):
    # +inf outside the unit box (the fit's score of inadmissible theta)
    if np.any(np.abs(x) > 1.0):
        return math.inf
    return float(np.sum((x - 0.25) ** 2) + 0.1 * x[0] * x[-1])


CASES = [
    (rosenbrock, [-1.2, 1.0], 0.5, dict(ftol=1e-10, xtol=1e-8, max_iter=1000)),
    (rosenbrock, [0.0, 0.0, 0.0], 1.0, dict(ftol=1e-9, xtol=1e-7, max_iter=2000)),
    (weighted_quadratic, [1.0, -2.0, 0.5, 3.0], 1.0, {}),
    (weighted_quadratic, [0.0], 1.0, dict(ftol=1e-12, xtol=1e-10)),
    (weighted_quadratic, [0.0] * 8, [0.5] * 8, dict(ftol=1e-10, xtol=1e-6, max_iter=4000)),
    (boxed, [0.9, -0.9, 0.5], 0.8, dict(ftol=1e-9, xtol=1e-6)),
    (rosenbrock, [0.0, 0.0], 1.0, dict(max_iter=20)),                # stops at the cap
]


@pytest.mark.parametrize("f,x0,step,kw", CASES)
def test_same_path_as_the_oracle(f, x0, step, kw):
    x, fv, it, nev, st = hmle.nelder_mead(f, x0, step, **kw)
    xo, fo, ito, nevo = oracle.nelder_mead(f, x0, step, **kw)
    assert (it, nev) == (ito, nevo)
    assert np.abs(x - xo).max() <= 1e-12 * max(1.0, np.abs(xo).max())
    assert abs(fv - fo) <= 1e-12 * max(1.0, abs(fo))
    assert st == (7 if it >= kw.get("max_iter", 400) else 0)


def test_reaches_the_known_minima():
    x, fv, it, nev, st = hmle.nelder_mead(rosenbrock, [-1.2, 1.0], 0.5,
                                          ftol=1e-14, xtol=1e-10, max_iter=2000)
    assert st == 0 and np.abs(x - 1.0).max() <= 1e-6 and fv <= 1e-12
    x, fv, it, nev, st = hmle.nelder_mead(weighted_quadratic, [1.0, -2.0, 0.5], 1.0,
                                          ftol=1e-14, xtol=1e-10)
    assert st == 0 and np.abs(x - 0.3).max() <= 1e-6


def test_nan_counts_as_infinity():
    g = lambda x: math.nan if x[0] > 0.8 else float((x[0] - 0.5) ** 2 + (x[1] + 0.2) ** 2)
    h = lambda x: math.inf if x[0] > 0.8 else g(x)
    a = hmle.nelder_mead(g, [0.0, 0.0], 1.0, ftol=1e-12, xtol=1e-9)
    b = hmle.nelder_mead(h, [0.0, 0.0], 1.0, ftol=1e-12, xtol=1e-9)
    assert (a[2], a[3]) == (b[2], b[3]) and np.array_equal(a[0], b[0])
    assert np.abs(a[0] - [0.5, -0.2]).max() <= 1e-6


@pytest.mark.parametrize("x0", [[], [0.0] * 9])
def test_rejects_bad_dimensions(x0):
    with pytest.raises(hmle.HmleError) as e:
        hmle.nelder_mead(weighted_quadratic, x0)
    assert e.value.status == 1


def test_rejects_non_finite_start():
    with pytest.raises(hmle.HmleError) as e:
        hmle.nelder_mead(weighted_quadratic, [0.0, math.nan])
    assert e.value.status == 1
