"""Observables of a parallel-tempering run (Sec. 5.1 of the paper) from the
measured energy and magnetisation series of its temperature slots.

- <E>/L and <M> per slot;
- the fourth-order energy cumulant U_E = <E^4> / <E^2>^2 (Eq. 11);
- the Binder cumulant V_M = 1 - <M^4> / (3 <M^2>^2) (Eq. 12);
each with a jackknife error (the paper's error method, Sec. 5.1): the series
is cut into `nblocks` consecutive blocks, every estimator is re-evaluated with
one block left out, and the error is sqrt((n-1)/n sum_b (theta_b - mean
theta)^2).  All estimators here are functions of sample means of powers of E
and M, so a leave-one-block-out estimate is taken from (total - block) power
sums: O(samples + blocks) work for every slot at once.
"""
import numpy as np

_POWERS = (1, 2, 4)


def _power_means(x, nblocks):
    """Means of x^p over the whole (truncated) series and with each block left
    out: dicts p -> [R] and p -> [nblocks, R]."""
    x = np.asarray(x, dtype=np.float64)
    if x.ndim == 1:
        x = x[:, None]
    n = (x.shape[0] // nblocks) * nblocks
    if n == 0:
        raise ValueError("need at least %d samples" % nblocks)
    size = n // nblocks
    xb = x[:n].reshape(nblocks, size, x.shape[1])
    full, loo = {}, {}
    for p in _POWERS:
        bs = (xb ** p).sum(axis=1)  # [nblocks, R]
        tot = bs.sum(axis=0)
        full[p] = tot / n
        loo[p] = (tot[None, :] - bs) / (n - size)
    return full, loo


def _jk(f, full, loo):
    theta = f(full)
    tb = f(loo)
    nb = tb.shape[0]
    err = np.sqrt((nb - 1) / nb * ((tb - tb.mean(axis=0)) ** 2).sum(axis=0))
    return theta, err


def observables(E, M, L, nblocks=20):
    """E, M: [samples, slots] series (slot order).  Returns a dict of [slots]
    arrays: e, e_err (<E>/L), m, m_err (<M>), UE, UE_err (Eq. 11), VM, VM_err
    (Eq. 12)."""
    fe, le = _power_means(E, nblocks)
    fm, lm = _power_means(M, nblocks)
    out = {}
    out["e"], out["e_err"] = _jk(lambda d: d[1] / L, fe, le)
    out["m"], out["m_err"] = _jk(lambda d: d[1], fm, lm)
    out["UE"], out["UE_err"] = _jk(lambda d: d[4] / (d[2] * d[2]), fe, le)
    out["VM"], out["VM_err"] = _jk(lambda d: 1.0 - d[4] / (3.0 * d[2] * d[2]), fm, lm)
    return out
