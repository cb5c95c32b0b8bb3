"""Near ties on the GPU, through the C ABI, against the oracle.

A near tie is a decision whose FP64 margin |beta dE + ln u| (Metropolis,
Eq. 8) or |D - ln u| (exchange, Eq. 9) is below 1e-9; there the GPU's exp and
log and the host's may round to different decisions.  These tests put such
decisions where they want them: from the initial configuration (the same on
both sides) and the known Philox draws, each slot's temperature is chosen so
that its first attempt sits at margin ~0 (or, for the exchange, each stage-0
pair's temperatures so that the first exchange does).  Then:
  - the GPU counts exactly those ties and logs them where they fell (slot,
    sweep, attempt / pair, exchange index, stage), as the oracle does;
  - the oracle, given the GPU's log, adopts the GPU's decision at each of them
    (and only there), and the two trajectories stay bit-identical for the rest
    of the run (the re-synchronisation reading of Eq. 8 and Eq. 9).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1308_5426_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def plr():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1308_5426_gb300
    return paper_1308_5426_gb300


def _draw_metro(seed, k, t, n, q, a):
    x = oracle.philox4x32_10([k, t, n, 1], [seed & 0xFFFFFFFF, seed >> 32])
    b = (a + 1 + ((int(x[0]) * (q - 1)) >> 32)) % q
    u = ((((int(x[1]) << 32) | int(x[2])) >> 11) + 1) * 2.0 ** -53
    return b, u


def _draw_exch(seed, t, stage, m):
    x = oracle.philox4x32_10([t, stage, m, 2], [seed & 0xFFFFFFFF, seed >> 32])
    return ((((int(x[1]) << 32) | int(x[2])) >> 11) + 1) * 2.0 ** -53


def _resync(g, o):
    """Hand the oracle every decision the GPU took at a near tie so far."""
    ev, n = g.near_log()
    assert n <= len(ev)  # nothing dropped from the log
    o.set_overrides(ev)
    return ev


def _check_equal(g, o, what):
    np.testing.assert_array_equal(g.spins(), o.spins(), err_msg=what)
    E, M = g.measure()
    Eo = o.energy()
    np.testing.assert_allclose(E, Eo, rtol=1e-10, atol=1e-10 * np.abs(Eo).max(), err_msg=what)
    np.testing.assert_allclose(M, o.magnetisation(), rtol=0, atol=1e-14, err_msg=what)
    np.testing.assert_allclose(g.running_energy(), o.running_energy(), rtol=1e-10,
                               atol=1e-10 * np.abs(Eo).max(), err_msg=what)
    gs, st = g.stats(), o.stats()
    np.testing.assert_array_equal(gs["acc_flip"], st["acc_flip"], err_msg=what)
    np.testing.assert_array_equal(gs["acc_swap"], st["acc_swap"], err_msg=what)
    assert gs["near_metro"] == int(st["near_metro"].sum()) and gs["near_exch"] == st["near_exch"], what


def _events(log):
    return sorted(tuple(int(v) for v in row[:4]) for row in log)


@pytest.mark.parametrize("precision,variant", [("fp64", "auto"), ("fx64", "auto"), ("fp64", "direct"),
                                               ("fp64", "global")])
def test_metropolis_ties_logged_and_resynchronised(plr, precision, variant):
    L, q, sigma, R, seed = 64, 3, 0.5, 32, 5
    temps0 = workloads.geometric_ratios(R, 0.05, 1.0) * oracle.jtot(L, sigma)
    o0 = oracle.Oracle(L, q, sigma, temps0, seed)
    S, h = o0.spins(), o0.fields()
    T = temps0.copy()
    tied = []
    for t in range(R):
        a = int(S[t, 0])
        b, u = _draw_metro(seed, 0, t, 0, q, a)
        dE = 2.0 * (h[t, a, 0] - h[t, b, 0])
        if dE > 0:  # only then does u decide
            T[t] = dE / -math.log(u)
            tied.append(t)
    assert len(tied) >= 4
    g = plr.Job(L, q, sigma, T, seed, precision=precision, sweep_variant=variant)
    direct = variant == "direct"
    o = oracle.Oracle(L, q, sigma, T, seed, fields=not direct)
    mode = "direct" if direct else "field"
    np.testing.assert_array_equal(g.spins(), o.spins())
    for n in range(40):
        g.sweep(1)
        ev = _resync(g, o)
        o.sweep(1, mode=mode)
        if n == 0:
            # exactly the constructed ties, on both sides, where they were put
            assert _events(ev) == [(0, t, 0, 0) for t in tied]
            olog, on = o.near_log()
            assert on == len(tied) and _events(olog) == _events(ev)
            np.testing.assert_array_equal(g.spins(), o.spins())
        g.exchange()
        _resync(g, o)
        o.exchange()
    _check_equal(g, o, "%s %s after 40 steps across %d ties" % (precision, variant, len(tied)))
    ad = o.adopted()
    assert int(ad["metro"].sum()) == len(tied)  # the oracle took the GPU's decision at every tie
    olog, _ = o.near_log()
    reversed_ = int(ad["metro_reversed"].sum())
    print("%s %s: %d ties, the GPU decided %d of them differently from the host"
          % (precision, variant, len(tied), reversed_))
    g.close()


@pytest.mark.parametrize("precision", ["fp64", "fx64"])
def test_exchange_ties_logged_and_resynchronised(plr, precision):
    """Ties at the first exchange (before any sweep), one per stage-0 pair."""
    L, q, sigma, R, seed = 64, 4, 0.7, 24, 6
    temps0 = workloads.geometric_ratios(R, 0.05, 1.0) * oracle.jtot(L, sigma)
    E = oracle.Oracle(L, q, sigma, temps0, seed).running_energy()
    beta = 1.0 / temps0
    T = temps0.copy()
    tied = []
    for t in range(0, R - 1, 2):
        u = _draw_exch(seed, t, 0, 0)
        dE = E[t] - E[t + 1]
        if dE == 0.0:
            continue
        b1 = beta[t] - math.log(u) / dE  # (beta_t - b1) dE = ln u
        if b1 > 0:
            T[t + 1] = 1.0 / b1
            tied.append(t)
    assert len(tied) >= 3
    g = plr.Job(L, q, sigma, T, seed, precision=precision)
    o = oracle.Oracle(L, q, sigma, T, seed)
    g.exchange()
    ev = _resync(g, o)
    o.exchange()
    assert _events(ev) == [(1, t, 0, 0) for t in tied]
    olog, on = o.near_log()
    assert on == len(tied) and _events(olog) == _events(ev)
    _check_equal(g, o, "%s after the tied exchange" % precision)
    for _ in range(30):
        g.sweep(1)
        _resync(g, o)
        o.sweep(1)
        g.exchange()
        _resync(g, o)
        o.exchange()
    _check_equal(g, o, "%s 30 steps after the tied exchange" % precision)
    assert o.adopted()["exch"] == len(tied)
    g.close()


def test_log_needs_valid_arguments(plr):
    import ctypes
    from paper_1308_5426_gb300 import _lib
    lib = _lib.load()
    g = plr.Job(32, 2, 0.5, np.ones(2), 1)
    n = ctypes.c_int(-1)
    assert lib.potts_lr_near_log(g.handle, None, 0, ctypes.byref(n)) == _lib.OK and n.value == 0
    assert lib.potts_lr_near_log(g.handle, None, 4, ctypes.byref(n)) == _lib.EINVAL
    assert lib.potts_lr_near_log(g.handle, None, -1, ctypes.byref(n)) == _lib.EINVAL
    assert lib.potts_lr_near_log(g.handle, None, 0, None) == _lib.EINVAL
    g.close()
