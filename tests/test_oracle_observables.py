"""Pins of the observables of Sec. 5.1 (Eq. 11, Eq. 12) and of the jackknife,
and the library's analysis module against them."""
import math

import numpy as np
import pytest

from oracle import Oracle
from oracle.enumerate import exact_averages
from oracle.jstar import jstar, jtot
from oracle.observables import binder_cumulant, energy_cumulant, jackknife, mean


def test_cumulants_closed_forms():
    """Three-point law {-a, 0, a} with weights (p/2, 1-p, p/2): U = 1/p;
    two-point +-a: U = 1; constant M: V = 2/3; M in {0, 1} with fraction p of
    ones: V = 1 - 1/(3p)."""
    a = 3.7
    E = [-a] * 10 + [0.0] * 60 + [a] * 10  # p = 0.25
    assert energy_cumulant(E) == pytest.approx(4.0, rel=1e-14)
    assert energy_cumulant([-a, a] * 7) == pytest.approx(1.0, rel=1e-14)
    assert binder_cumulant([0.42] * 9) == pytest.approx(2.0 / 3.0, rel=1e-14)
    M = [1.0] * 30 + [0.0] * 70
    assert binder_cumulant(M) == pytest.approx(1.0 - 1.0 / (3 * 0.3), rel=1e-14)


def test_jackknife_of_the_mean_is_the_standard_error_of_block_means():
    """For the (linear) sample mean the jackknife error equals the standard
    error of the block means exactly."""
    rng = np.random.default_rng(3)
    x = list(rng.normal(size=1000))
    nb = 20
    est, err = jackknife(x, mean, nb)
    bm = np.array(x).reshape(nb, -1).mean(axis=1)
    se = math.sqrt(((bm - bm.mean()) ** 2).sum() / (nb * (nb - 1)))
    assert est == pytest.approx(np.mean(x), rel=1e-13)
    assert err == pytest.approx(se, rel=1e-12)


def test_cumulants_of_the_oracle_chain_match_exact_enumeration():
    """U_E and V_M per slot of the oracle's PT chain at L=8, q=3 agree with
    their exact values (from <E^2>, <E^4>, <M^2>, <M^4> by enumeration of
    all 3^8 states) within 3 jackknife errors."""
    L, q, sigma, c = 8, 3, 0.5, 2
    ratios = np.array([0.15, 0.3, 0.6])
    temps = ratios * jtot(L, sigma)
    o = Oracle(L, q, sigma, temps, seed=99, c=c)
    for _ in range(500):
        o.step()
    n = 40_000
    E = np.zeros((n, o.R))
    M = np.zeros((n, o.R))
    for k in range(n):
        o.step()
        E[k] = o.running_energy()
        M[k] = o.magnetisation()
    ex = exact_averages(L, q, jstar(L, sigma), c, 1.0 / temps)
    for t in range(o.R):
        ue, ue_err = jackknife(list(E[:, t]), energy_cumulant, 40)
        vm, vm_err = jackknife(list(M[:, t]), binder_cumulant, 40)
        ue_x = ex["E4"][t] / ex["E2"][t] ** 2
        vm_x = 1.0 - ex["M4"][t] / (3.0 * ex["M2"][t] ** 2)
        assert abs(ue - ue_x) < 3 * ue_err + 1e-6, (t, ue, ue_x, ue_err)
        assert abs(vm - vm_x) < 3 * vm_err + 1e-6, (t, vm, vm_x, vm_err)


def test_library_analysis_equals_the_definitions():
    """paper_1308_5426_gb300.analysis (vectorised leave-one-block-out sums)
    gives the definitions' estimates and jackknife errors."""
    from paper_1308_5426_gb300.analysis import observables
    rng = np.random.default_rng(11)
    n, R, L, nb = 600, 3, 50, 12
    E = -L * (1.0 + 0.3 * rng.random((n, R)))
    M = rng.random((n, R))
    got = observables(E, M, L, nb)
    for t in range(R):
        e, e_err = jackknife(list(E[:, t]), lambda xs: mean(xs) / L, nb)
        m, m_err = jackknife(list(M[:, t]), mean, nb)
        ue, ue_err = jackknife(list(E[:, t]), energy_cumulant, nb)
        vm, vm_err = jackknife(list(M[:, t]), binder_cumulant, nb)
        for key, ref in (("e", e), ("e_err", e_err), ("m", m), ("m_err", m_err), ("UE", ue),
                         ("UE_err", ue_err), ("VM", vm), ("VM_err", vm_err)):
            assert got[key][t] == pytest.approx(ref, rel=1e-9, abs=1e-14), (key, t)
