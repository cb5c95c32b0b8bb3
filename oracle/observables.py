"""Observables of Sec. 5.1 and their jackknife errors, from the definitions.

TEST INFRASTRUCTURE (see oracle/__init__.py): only tests, the smoke check and
the benchmark's CPU legs use this module.  Each function is the plain textbook
formula, evaluated with loops and no shortcuts, so that it can be checked by
eye; the library's own analysis module computes the same quantities
independently.

- Fourth-order energy cumulant, Eq. 11: U_E = <E^4> / <E^2>^2.
- Binder cumulant of the magnetisation, Eq. 12: V_M = 1 - <M^4> / (3 <M^2>^2).
- Jackknife (the error method the paper takes from ALPS, Sec. 5.1): the series
  is cut into n consecutive blocks of equal length; theta_b is the estimator
  evaluated on the series with block b left out; the estimate of the error is
  sqrt((n - 1) / n * sum_b (theta_b - mean_b theta_b)^2).
"""
import math


def mean(xs):
    return sum(xs) / len(xs)


def energy_cumulant(E):
    """U_E^(4) = <E^4> / <E^2>^2 over the samples E (Eq. 11)."""
    e2 = mean([e * e for e in E])
    e4 = mean([e ** 4 for e in E])
    return e4 / (e2 * e2)


def binder_cumulant(M):
    """V_M^(4) = 1 - <M^4> / (3 <M^2>^2) over the samples M (Eq. 12)."""
    m2 = mean([m * m for m in M])
    m4 = mean([m ** 4 for m in M])
    return 1.0 - m4 / (3.0 * m2 * m2)


def jackknife(series, estimator, nblocks):
    """(estimate on the whole series, jackknife error) of estimator(series)
    with nblocks leave-one-block-out estimates; the series is truncated to a
    multiple of nblocks."""
    n = len(series) // nblocks * nblocks
    xs = list(series[:n])
    size = n // nblocks
    thetas = []
    for b in range(nblocks):
        kept = xs[: b * size] + xs[(b + 1) * size:]
        thetas.append(estimator(kept))
    tbar = mean(thetas)
    var = (nblocks - 1) / nblocks * sum((t - tbar) ** 2 for t in thetas)
    return estimator(xs), math.sqrt(var)
