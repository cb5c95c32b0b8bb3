"""The precision contract at the precision workload's full size: L = 4096,
q = 8, sigma = 0.2, R = 128 temperatures geometric in T/Jtot in [0.02, 0.5],
seed 1.  FP32 fields with the split-BF16 tensor-core rebuild (longest
interval K = 100 sweeps) against plain FP64 fields, same seed and call
sequence:
  - the FP32 field drift, max |h32 - h64| / Jtot over all slots, states and
    sites (h64 the FP64 direct sums of the same spins), stays below 1e-5 at
    every check, one every 10 sweeps over the whole run;
  - after 500 sweeps of warm-up, <E>/L and <M> of every slot over 2000 sweeps
    (measured every sweep, 20 bins of 100 sweeps) agree within 3 combined
    binned standard errors; slots frozen in an ordered state (standard error
    zero on both sides) must agree exactly.
Each slot's difference and its ratio to the combined standard error are
printed (the error of each FP32 result against FP64)."""
import math

import numpy as np
import pytest

import oracle
from paper_1308_5426_gb300 import workloads

pytestmark = pytest.mark.gpu

WARM, PROD, NBINS, CHECK_EVERY = 500, 2000, 20, 10


@pytest.fixture(scope="module")
def plr():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1308_5426_gb300
    return paper_1308_5426_gb300


def _binned(x, nbins):
    """Mean and binned standard error of each column of x (rows in time order)."""
    n = (x.shape[0] // nbins) * nbins
    b = x[:n].reshape(nbins, -1, x.shape[1]).mean(axis=1)
    return b.mean(axis=0), b.std(axis=0, ddof=1) / math.sqrt(nbins)


def _run(plr, spec, precision):
    L, R = spec.L, spec.R
    temps = spec.ratios * oracle.jtot(L, spec.sigma)
    j = plr.Job(L, spec.q, spec.sigma, temps, spec.seed, precision=precision, recompute_every=100)
    drift = []
    for n in range(WARM):
        j.sweep(1)
        j.exchange()
        if precision == "fp32" and (n + 1) % CHECK_EVERY == 0:
            drift.append(j.fields_error())
    E = np.zeros((PROD, R))
    M = np.zeros((PROD, R))
    for n in range(PROD):
        j.sweep(1)
        j.exchange()
        E[n], M[n] = j.measure()
        if precision == "fp32" and (n + 1) % CHECK_EVERY == 0:
            drift.append(j.fields_error())
    j.close()
    return E / L, M, np.array(drift)


def test_fp32_against_fp64_at_the_precision_workload(plr):
    spec = workloads.precision_job("fp32")
    assert (spec.L, spec.q, spec.sigma, spec.R, spec.seed) == (4096, 8, 0.2, 128, 1)
    E32, M32, drift = _run(plr, spec, "fp32")
    E64, M64, _ = _run(plr, spec, "fp64")
    assert drift.size == (WARM + PROD) // CHECK_EVERY
    print("FP32 field drift over %d checks: max %.3e Jtot" % (drift.size, drift.max()))
    assert drift.max() < 1e-5, drift.max()
    for name, a, b in (("E/L", E32, E64), ("M", M32, M64)):
        ma, sa = _binned(a, NBINS)
        mb, sb = _binned(b, NBINS)
        se = np.hypot(sa, sb)
        diff = ma - mb
        frozen = se <= 1e-12 * np.maximum(np.abs(mb), 1.0)
        z = np.where(frozen, 0.0, diff / np.where(frozen, 1.0, se))
        print("%s: %d frozen slots, max |FP32 - FP64| %.3e, max |diff|/SE %.2f, mean (diff/SE)^2 %.2f"
              % (name, frozen.sum(), np.abs(diff).max(), np.abs(z).max(), float((z[~frozen] ** 2).mean())))
        for t in range(spec.R):
            print("  slot %3d %s fp32 %.6f fp64 %.6f se %.2e z %+.2f" % (t, name, ma[t], mb[t], se[t], z[t]))
        np.testing.assert_allclose(ma[frozen], mb[frozen], rtol=1e-12, atol=0, err_msg=name + " frozen slots")
        bad = np.nonzero(np.abs(diff) >= 3 * se + 1e-12)[0]
        assert bad.size == 0, (name, bad, diff[bad], se[bad])
