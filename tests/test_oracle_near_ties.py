"""Pins of the oracle's near-tie accounting and of its re-synchronisation.

A near tie is a decision whose FP64 margin |beta dE + ln u| (Metropolis, Eq. 8)
or |D - ln u| (exchange, Eq. 9) is below 1e-9.  These tests construct such
decisions on purpose: from a known state and the known Philox draw of one
proposal (or one exchange pair), they pick the temperature that puts the
margin at a chosen value, then check that the oracle counts, dates and logs
exactly those decisions, that the 1e-9 bound sits where it should (both
signs), and that a tabled decision is adopted at a counted tie -- and only
there.  A construction error (wrong draw, wrong sign) would leave no tie to
count, so it fails these tests rather than passing them.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1308_5426_gb300 import workloads

L, Q, SIGMA, R, SEED = 48, 4, 0.6, 8, 17
N0 = 3  # the constructed decisions come at sweep (and exchange) index 3


def _draw_metro(seed, k, t, n, q, a):
    """Proposal b and u of attempt k of slot t at sweep n (the counter layout
    and value maps stated in the oracle's header)."""
    x = oracle.philox4x32_10([k, t, n, 1], [seed & 0xFFFFFFFF, seed >> 32])
    b = (a + 1 + ((int(x[0]) * (q - 1)) >> 32)) % q
    u = ((((int(x[1]) << 32) | int(x[2])) >> 11) + 1) * 2.0 ** -53
    return b, u


def _draw_exch(seed, t, stage, m):
    x = oracle.philox4x32_10([t, stage, m, 2], [seed & 0xFFFFFFFF, seed >> 32])
    return ((((int(x[1]) << 32) | int(x[2])) >> 11) + 1) * 2.0 ** -53


def _state_after(steps):
    temps = workloads.geometric_ratios(R, 0.05, 1.0) * oracle.jtot(L, SIGMA)
    o = oracle.Oracle(L, Q, SIGMA, temps, SEED)
    for _ in range(steps):
        o.step()
    return temps, o.spins()


def _restart(temps, S):
    """A fresh oracle holding configuration S at sweep and exchange index N0
    (fields and energies recomputed from S by the plain sums)."""
    o = oracle.Oracle(L, Q, SIGMA, temps, SEED)
    o.set_spins(S)
    o.set_counters(N0, N0)
    return o


def _metro_tie(delta=0.0):
    """Temperatures that put the first attempt of sweep N0 in the first slot
    with dE > 0 at margin beta dE + ln u = delta; returns (temps, S, t, a, b)."""
    temps, S = _state_after(N0)
    h = _restart(temps, S).fields()
    for t in range(R):
        a = int(S[t, 0])
        b, u = _draw_metro(SEED, 0, t, N0, Q, a)
        dE = 2.0 * (h[t, a, 0] - h[t, b, 0])  # c = 2
        if dE > 0:
            T = temps.copy()
            T[t] = dE / (-math.log(u) + delta)
            return T, S, t, a, b
    pytest.skip("no slot with dE > 0 at the first site")


def _exch_tie(delta=0.0):
    """Temperatures that put exchange N0, stage 0, pair (t, t+1) at margin
    D - ln u = delta; returns (temps, S, t)."""
    temps, S = _state_after(N0)
    E = _restart(temps, S).running_energy()
    beta = 1.0 / temps
    for t in range(0, R - 1, 2):
        u = _draw_exch(SEED, t, 0, N0)
        dE = E[t] - E[t + 1]
        if dE == 0.0:
            continue
        b1 = beta[t] - (math.log(u) + delta) / dE
        if b1 > 0:
            T = temps.copy()
            T[t + 1] = 1.0 / b1
            return T, S, t
    pytest.skip("no stage-0 pair admits a positive temperature")


def test_metropolis_tie_is_counted_dated_and_logged():
    T, S, t, a, b = _metro_tie()
    o = _restart(T, S)
    o.sweep(1)
    st = o.stats()
    expect = np.zeros(R, np.uint64)
    expect[t] = 1
    np.testing.assert_array_equal(st["near_metro"], expect)
    assert st["first_near_metro"][t] == N0
    assert all(st["first_near_metro"][s] == -1 for s in range(R) if s != t)
    assert st["near_exch"] == 0
    log, n = o.near_log()
    assert n == 1
    kind, slot, idx, attempt, own, taken = log[0].tolist()
    assert (kind, slot, idx, attempt) == (0, t, N0, 0)
    assert own == taken
    # the decision the log reports is the one the configuration shows
    assert int(o.spins()[t, 0]) == (b if own else a)


@pytest.mark.parametrize("delta,counted", [(5e-10, True), (-5e-10, True), (2e-9, False), (-2e-9, False)])
def test_metropolis_tie_bound(delta, counted):
    """The bound is |beta dE + ln u| < 1e-9, on both sides of zero."""
    T, S, t, _, _ = _metro_tie(delta)
    o = _restart(T, S)
    o.sweep(1)
    assert int(o.stats()["near_metro"][t]) == (1 if counted else 0)


def test_exchange_tie_is_counted_dated_and_logged():
    T, S, t = _exch_tie()
    o = _restart(T, S)
    E0 = o.running_energy()
    o.exchange()
    st = o.stats()
    assert st["near_exch"] == 1 and st["first_near_exch"] == N0
    assert int(st["near_metro"].sum()) == 0
    log, n = o.near_log()
    assert n == 1
    kind, pair, idx, stage, own, taken = log[0].tolist()
    assert (kind, pair, idx, stage) == (1, t, N0, 0) and own == taken
    # the energies show whether the pair swapped
    E1 = o.running_energy()
    assert (E1[t] == E0[t + 1] and E1[t + 1] == E0[t]) == bool(own)


@pytest.mark.parametrize("delta,counted", [(5e-10, True), (-5e-10, True), (2e-9, False), (-2e-9, False)])
def test_exchange_tie_bound(delta, counted):
    T, S, _ = _exch_tie(delta)
    o = _restart(T, S)
    o.exchange()
    assert o.stats()["near_exch"] == (1 if counted else 0)


def test_adopted_decision_reverses_the_oracle_and_the_chain_stays_consistent():
    """A tabled decision at a counted tie is taken even where it reverses the
    oracle's own; the fields and energies then follow the adopted move, and a
    direct-sum oracle given the same table follows the same trajectory."""
    T, S, t, a, b = _metro_tie()
    probe = _restart(T, S)
    probe.sweep(1)
    own = int(probe.near_log()[0][0][4])
    table = [[0, t, N0, 0, 1 - own]]
    f = _restart(T, S)
    f.set_overrides(table)
    d = oracle.Oracle(L, Q, SIGMA, T, SEED, fields=False)
    d.set_spins(S)
    d.set_counters(N0, N0)
    d.set_overrides(table)
    f.sweep(1)
    d.sweep(1, mode="direct")
    ad = f.adopted()
    assert int(ad["metro"][t]) == 1 and int(ad["metro_reversed"][t]) == 1
    assert int(ad["metro"].sum()) == 1 and ad["exch"] == 0
    assert int(f.spins()[t, 0]) == (b if 1 - own else a)
    assert int(probe.spins()[t, 0]) != int(f.spins()[t, 0])  # the reversal took effect
    np.testing.assert_array_equal(f.spins(), d.spins())
    assert int(d.adopted()["metro"][t]) == 1
    for _ in range(20):
        f.step()
        d.step(mode="direct")
    np.testing.assert_array_equal(f.spins(), d.spins())
    # the adopted move entered the fields and the energy exactly as a move does
    jt = oracle.jtot(L, SIGMA)
    fresh = oracle.Oracle(L, Q, SIGMA, T, SEED)
    fresh.set_spins(f.spins())
    np.testing.assert_allclose(f.fields(), fresh.fields(), rtol=0, atol=1e-12 * jt)
    np.testing.assert_allclose(f.running_energy(), f.energy(), rtol=1e-10)


def test_table_is_not_consulted_away_from_ties():
    """An entry for a decision that is not a near tie changes nothing."""
    temps, S = _state_after(N0)
    plain = _restart(temps, S)
    plain.sweep(2)
    tabled = _restart(temps, S)
    # contradictory entries for every first attempt of sweep N0 (none of them is a tie)
    tabled.set_overrides([[0, t, N0, 0, 0] for t in range(R)] + [[0, t, N0, 0, 1] for t in range(R)])
    tabled.sweep(2)
    np.testing.assert_array_equal(tabled.spins(), plain.spins())
    ad = tabled.adopted()
    assert int(ad["metro"].sum()) == 0 and ad["exch"] == 0


def test_adopted_exchange_decision():
    T, S, t = _exch_tie()
    probe = _restart(T, S)
    E0 = probe.running_energy()
    probe.exchange()
    own = int(probe.near_log()[0][0][4])
    o = _restart(T, S)
    o.set_overrides([[1, t, N0, 0, 1 - own]])
    o.exchange()
    ad = o.adopted()
    assert ad["exch"] == 1 and ad["exch_reversed"] == 1
    E1 = o.running_energy()
    assert (E1[t] == E0[t + 1] and E1[t + 1] == E0[t]) == bool(1 - own)
    st = o.stats()
    assert int(st["acc_swap"][t]) == (1 - own)
