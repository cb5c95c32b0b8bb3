"""Pins of the oracle's energy, magnetisation and field bookkeeping (Eq. 2,
Eq. 10) against closed forms and a second, independent way of counting."""
import math

import numpy as np
import pytest

from oracle import Oracle
from oracle.jstar import jstar, jtot


def _oracle_with(L, q, sigma, spins, c=2, T=1.0):
    R = spins.shape[0]
    o = Oracle(L, q, sigma, np.full(R, T), seed=3, c=c)
    o.set_spins(spins)
    return o


@pytest.mark.parametrize("c", [1, 2])
def test_worked_example_sigma_one(c):
    """L = 4, sigma = 1: J*(1) = J*(3) = pi^2/8, J*(2) = pi^2/16 (closed form of
    Eq. 5).  Spins (0,0,1,1): equal pairs at distance 1 -> E = -(c/2) 4 J*(1);
    spins (0,1,0,1): equal pairs at distance 2 -> E = -(c/2) 4 J*(2); all equal:
    E = -(c/2) * 4 * (2 J*(1) + J*(2))."""
    S = np.array([[0, 0, 1, 1], [0, 1, 0, 1], [1, 1, 1, 1]], dtype=np.uint8)
    o = _oracle_with(4, 2, 1.0, S, c=c)
    j1, j2 = math.pi ** 2 / 8, math.pi ** 2 / 16
    ref = np.array([-0.5 * c * 4 * j1, -0.5 * c * 4 * j2, -0.5 * c * 4 * (2 * j1 + j2)])
    np.testing.assert_allclose(o.energy(), ref, rtol=1e-14)
    np.testing.assert_allclose(o.running_energy(), ref, rtol=1e-14)
    np.testing.assert_allclose(o.magnetisation(), [0.0, 0.0, 1.0])


@pytest.mark.parametrize("L,q,sigma", [(64, 3, 0.5), (1000, 5, 0.4), (37, 16, 0.1), (2, 2, 0.5), (3, 16, 2.0)])
@pytest.mark.parametrize("c", [1, 2])
def test_ground_state(L, q, sigma, c):
    """Ordered configuration: E_gs = -(c/2) L Jtot, M = 1 (Eq. 2, Eq. 10)."""
    S = np.stack([np.full(L, x % q, dtype=np.uint8) for x in range(3)])
    o = _oracle_with(L, q, sigma, S, c=c)
    np.testing.assert_allclose(o.energy(), -0.5 * c * L * jtot(L, sigma), rtol=1e-12)
    np.testing.assert_allclose(o.magnetisation(), 1.0)


@pytest.mark.parametrize("L,q", [(60, 3), (64, 4), (45, 5)])
def test_magnetisation_balanced(L, q):
    """Equal occupation of all q states gives M = 0 (Eq. 10)."""
    S = (np.arange(L) % q).astype(np.uint8)[None, :]
    o = _oracle_with(L, q, 0.5, S)
    if L % q == 0:
        assert o.magnetisation()[0] == pytest.approx(0.0, abs=1e-15)
    nmax = int(np.bincount(S[0], minlength=q).max())
    assert o.magnetisation()[0] == pytest.approx((q * nmax / L - 1) / (q - 1))


@pytest.mark.parametrize("L,q,sigma", [(64, 3, 0.5), (97, 7, 0.3), (256, 2, 0.9), (2, 2, 0.5), (3, 3, 1.0),
                                     (33, 16, 0.05)])
def test_energy_by_distance_counts(L, q, sigma):
    """Second route to Eq. 2: E = -(c/2) sum_r J*(r) N_r with N_r the number of
    ordered pairs at periodic offset r holding equal spins, counted by rolling
    the configuration.  Also Sum_x h[x][i] = Jtot and -(c/2) Sum_i h[s_i][i] = E
    for the oracle's fields."""
    rng = np.random.default_rng(11)
    S = rng.integers(0, q, size=(4, L)).astype(np.uint8)
    o = _oracle_with(L, q, sigma, S, c=2)
    J = jstar(L, sigma)
    # ordered pairs (i, j) with j - i = d (d = 1..L-1, not periodic) ... use |i-j| directly
    E_ref = []
    for s in S:
        e = 0.0
        for d in range(1, L):
            e += J[d] * 2 * np.count_nonzero(s[:-d] == s[d:])  # pairs (i, i+d) and (i+d, i)
        E_ref.append(-e)
    np.testing.assert_allclose(o.energy(), E_ref, rtol=1e-12)
    h = o.fields()
    np.testing.assert_allclose(h.sum(axis=1), jtot(L, sigma), rtol=1e-12)
    E_f = [-np.sum(h[t][S[t], np.arange(L)]) for t in range(4)]
    np.testing.assert_allclose(E_f, E_ref, rtol=1e-12)
