"""Pins of the oracle's Markov chain (Eq. 8, Eq. 9, Sec. 4.2) against exact
enumeration, limits with closed-form outcomes and exchange statistics."""
import math

import numpy as np
import pytest

from oracle import Oracle, philox4x32_10
from oracle.enumerate import exact_averages
from oracle.jstar import jstar, jtot


def _binned(x, nbins=50):
    x = np.asarray(x)
    b = x[: (x.size // nbins) * nbins].reshape(nbins, -1).mean(axis=1)
    return b.mean(), b.std(ddof=1) / math.sqrt(nbins)


@pytest.mark.parametrize("L,q,sigma,c,ratios", [
    (8, 3, 0.5, 2, (0.08, 0.15, 0.3, 0.6)),
    (10, 2, 0.8, 1, (0.1, 0.2, 0.4, 0.8)),
])
def test_pt_matches_exact_enumeration(L, q, sigma, c, ratios):
    """PT chains sample exp(-beta H): <E>, <E^2>, <M>, <M^2> per slot agree with
    exact enumeration over all q^L states within 3 binned standard errors."""
    J = jstar(L, sigma)
    temps = np.array(ratios) * jtot(L, sigma)
    o = Oracle(L, q, sigma, temps, seed=12345, c=c)
    burn, nmeas = 500, 60_000
    for _ in range(burn):
        o.step()
    E = np.zeros((nmeas, o.R))
    M = np.zeros((nmeas, o.R))
    for n in range(nmeas):
        o.step()
        E[n] = o.running_energy()
        M[n] = o.magnetisation()
    ex = exact_averages(L, q, J, c, 1.0 / temps)
    # the binned SE is floored by sqrt(Var/N) from the exact variance: a cold
    # slot that never leaves its ground state has a zero sample variance
    var = {"E": ex["E2"] - ex["E"] ** 2, "M": ex["M2"] - ex["M"] ** 2}
    for t in range(o.R):
        for name, series in (("E", E[:, t]), ("E2", E[:, t] ** 2), ("M", M[:, t]), ("M2", M[:, t] ** 2)):
            mean, se = _binned(series)
            base = name[0]
            scale = abs(2 * ex[base][t]) if name.endswith("2") else 1.0
            se = max(se, scale * math.sqrt(max(var[base][t], 0.0) / nmeas))
            assert abs(mean - ex[name][t]) < 3.0 * se + 1e-12, (t, name, mean, ex[name][t], se)
    st = o.stats()
    assert st["near_metro"].sum() == 0 and st["near_exch"] == 0
    assert np.all(st["acc_swap"] > 0)
    # running energy bookkeeping equals the plain double sum
    np.testing.assert_allclose(o.running_energy(), o.energy(), rtol=1e-11, atol=1e-11)


def test_infinite_temperature_follows_generator():
    """beta -> 0: every proposal is accepted (u <= 1 = exp(-0)), so one sweep
    maps s_k to b_k = (a + 1 + floor(x0 (q-1) / 2^32)) mod q with x0 the first
    Philox word of counter (k, t, 0, 1)."""
    L, q, R, seed = 50, 5, 3, 777
    o = Oracle(L, q, 0.5, np.full(R, 1e300), seed=seed)
    s0 = o.spins()
    o.sweep(1, mode="direct")
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint32)
    exp = s0.copy()
    for t in range(R):
        for k in range(L):
            x0 = int(philox4x32_10(np.array([k, t, 0, 1], np.uint32), key)[0])
            exp[t, k] = (int(exp[t, k]) + 1 + ((x0 * (q - 1)) >> 32)) % q
    np.testing.assert_array_equal(o.spins(), exp)
    assert o.stats()["acc_flip"].tolist() == [L] * R


def test_initial_spins_follow_generator():
    """Initial spins are floor(x0 q / 2^32) of Philox counter (i, t, 0, 0)."""
    L, q, R, seed = 40, 7, 2, 2**40 + 5
    o = Oracle(L, q, 0.3, np.ones(R), seed=seed)
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint32)
    exp = np.array([[(int(philox4x32_10(np.array([i, t, 0, 0], np.uint32), key)[0]) * q) >> 32
                     for i in range(L)] for t in range(R)], dtype=np.uint8)
    np.testing.assert_array_equal(o.spins(), exp)


@pytest.mark.parametrize("c", [1, 2])
def test_zero_temperature_ground_state_is_frozen(c):
    """beta -> infinity from the ordered state: every flip costs dE = c Jtot > 0,
    so nothing is ever accepted and E stays -(c/2) L Jtot."""
    L, q, sigma = 64, 4, 0.6
    o = Oracle(L, q, sigma, np.full(2, 1e-6), seed=5, c=c)
    o.set_spins(np.zeros((2, L), np.uint8))
    for _ in range(20):
        o.step(mode="direct")
    assert np.all(o.spins() == 0)
    assert o.stats()["acc_flip"].sum() == 0
    np.testing.assert_allclose(o.energy(), -0.5 * c * L * jtot(L, sigma), rtol=1e-12)


@pytest.mark.parametrize("c", [1, 2])
def test_infinite_temperature_mean_energy(c):
    """beta = 0: spins are uniform and independent, <E> = -(c/2) (L/q) Jtot."""
    L, q, sigma = 48, 3, 0.5
    o = Oracle(L, q, sigma, np.full(4, 1e300), seed=9, c=c)
    E = []
    for _ in range(3000):
        o.sweep(1)
        E.append(o.running_energy())
    E = np.array(E).ravel()
    mean, se = _binned(E)
    assert abs(mean - (-0.5 * c * L * jtot(L, sigma) / q)) < 3 * se


def test_field_mode_equals_direct_mode():
    """Incremental local fields and the direct O(L) sum give the same chain."""
    L, q, sigma = 64, 3, 0.5
    temps = np.geomspace(0.05, 1.0, 8) * jtot(L, sigma)
    a = Oracle(L, q, sigma, temps, seed=1)
    b = Oracle(L, q, sigma, temps, seed=1)
    for _ in range(200):
        a.step(mode="field")
        b.step(mode="direct")
    np.testing.assert_array_equal(a.spins(), b.spins())
    np.testing.assert_allclose(a.running_energy(), b.running_energy(), rtol=1e-11)
    np.testing.assert_allclose(a.fields().sum(axis=1), jtot(L, sigma), rtol=1e-11)
    assert a.stats()["near_metro"].sum() == 0


def test_exchange_acceptance_rate():
    """Two slots, no sweeps: from the state with D < 0 a swap is accepted with
    probability p = exp(D), after which D > 0 and the next swap always returns.
    The long-run accepted fraction is 2p / (1 + p) (Eq. 9); a flipped sign in D
    would give p = 1."""
    L, q, sigma = 16, 3, 0.5
    rng = np.random.default_rng(0)
    S = np.stack([np.zeros(L, np.uint8), rng.integers(0, q, L).astype(np.uint8)])
    o = Oracle(L, q, sigma, np.array([1.0, 3.0]), seed=4)
    o.set_spins(S)  # slot 0 (cold) holds the ground state: D < 0
    E = o.running_energy()
    D = (1.0 - 1.0 / 3.0) * (E[0] - E[1])
    assert D < 0
    p = math.exp(D)
    n = 40_000
    for _ in range(n):
        o.exchange()
    st = o.stats()
    frac = st["acc_swap"][0] / st["att_swap"][0]
    expect = 2 * p / (1 + p)
    assert abs(frac - expect) < 4 * math.sqrt(expect * (1 - expect) / n) + 1e-3, (frac, expect)


def _one_sweep_kernel(L, q, J, c, beta, rule):
    """Transition matrix of one sequential sweep (sites 0..L-1) over all q^L
    states, by brute force.  rule "metropolis" (Eq. 8): propose one of the
    other q-1 states uniformly, accept with min(1, exp(-beta dE)); rule
    "heatbath": draw the new state of the site from exp(-beta E) over all q."""
    import itertools
    states = list(itertools.product(range(q), repeat=L))
    index = {s: n for n, s in enumerate(states)}

    def energy(s):
        return -0.5 * c * sum(J[abs(i - j) % L] for i in range(L) for j in range(L) if i != j and s[i] == s[j])

    E = np.array([energy(s) for s in states])
    T = np.eye(len(states))
    for k in range(L):
        P = np.zeros_like(T)
        for n, s in enumerate(states):
            nbr = [index[s[:k] + (x,) + s[k + 1:]] for x in range(q)]
            if rule == "metropolis":
                for x in range(q):
                    if x == s[k]:
                        continue
                    p = min(1.0, math.exp(-beta * (E[nbr[x]] - E[n]))) / (q - 1)
                    P[n, nbr[x]] += p
                    P[n, n] += 1.0 / (q - 1) - p
            else:
                w = np.exp(-beta * (E[nbr] - E[nbr].min()))
                P[n, nbr] += w / w.sum()
        T = T @ P
    return T, index, E


def test_one_sweep_transition_law():
    """The oracle's sweep is the Metropolis chain of Eq. 8 with sequential sites
    and a uniform proposal: from a fixed start, the end states of many
    independent sweeps follow the brute-force one-sweep transition row (chi
    square), the Boltzmann weight is stationary under that matrix, and the same
    samples reject the heat-bath row (which has the same stationary law)."""
    from scipy.stats import chi2
    L, q, sigma, c = 4, 3, 0.5, 2
    J = jstar(L, sigma)
    ratios = np.array([0.15, 0.4, 1.0])
    temps = ratios * jtot(L, sigma)
    s0 = np.array([0, 1, 1, 2], dtype=np.uint8)
    o = Oracle(L, q, sigma, temps, seed=4242, c=c)
    nsamp = 20000
    counts = np.zeros((o.R, q ** L))
    for _ in range(nsamp):
        o.set_spins(np.tile(s0, (o.R, 1)))
        o.sweep(1, mode="direct")
        s = o.spins()
        for t in range(o.R):
            counts[t, int(sum(int(v) * q ** (L - 1 - i) for i, v in enumerate(s[t])))] += 1
    for t in range(o.R):
        beta = 1.0 / temps[t]
        T, index, E = _one_sweep_kernel(L, q, J, c, beta, "metropolis")
        pi = np.exp(-beta * (E - E.min()))
        pi /= pi.sum()
        np.testing.assert_allclose(pi @ T, pi, atol=1e-13)     # global balance of one sweep
        row = T[index[tuple(int(v) for v in s0)]]

        def stat(p):
            m = p * nsamp > 5
            x2 = ((counts[t][m] - nsamp * p[m]) ** 2 / (nsamp * p[m])).sum()
            return x2, int(m.sum()) - 1

        x2, dof = stat(row)
        assert chi2.sf(x2, dof) > 1e-4, (t, x2, dof)
        Th, _, _ = _one_sweep_kernel(L, q, J, c, beta, "heatbath")
        np.testing.assert_allclose(pi @ Th, pi, atol=1e-13)
        x2h, dofh = stat(Th[index[tuple(int(v) for v in s0)]])
        assert chi2.sf(x2h, dofh) < 1e-6, (t, x2h, dofh)


def test_random_site_order_follows_generator_at_infinite_temperature():
    """Random-site order, beta -> 0: attempt m of sweep n in slot t goes to site
    k = floor(x3 L / 2^32) of Philox counter (m, t, n, 3) and always flips it
    to (a + 1 + floor(x0 (q-1) / 2^32)) mod q, a being the site's current
    state (a site may be drawn twice in one sweep)."""
    L, q, R, seed = 40, 4, 2, 31
    o = Oracle(L, q, 1.0, np.full(R, 1e300), seed, site_order="random")
    s = o.spins().astype(np.int64)
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint32)
    for n in range(3):
        for t in range(R):
            for m in range(L):
                x = [int(v) for v in philox4x32_10(np.array([m, t, n, 3], np.uint32), key)]
                k = (x[3] * L) >> 32
                s[t, k] = (s[t, k] + 1 + ((x[0] * (q - 1)) >> 32)) % q
        o.sweep(1, mode="direct")
        np.testing.assert_array_equal(o.spins(), s)


def test_random_site_one_sweep_transition_law():
    """Random-site order is the chain of the averaged single-site kernel: one
    sweep = (1/L sum_k P_k)^L.  The oracle's end states from a fixed start
    follow that row (chi square), and reject the sequential-order row."""
    from scipy.stats import chi2
    L, q, sigma, c = 4, 3, 0.5, 2
    J = jstar(L, sigma)
    temps = np.array([0.2, 0.6]) * jtot(L, sigma)
    s0 = np.array([0, 1, 1, 2], dtype=np.uint8)
    o = Oracle(L, q, sigma, temps, seed=4343, c=c, site_order="random")
    nsamp = 20000
    counts = np.zeros((o.R, q ** L))
    for _ in range(nsamp):
        o.set_spins(np.tile(s0, (o.R, 1)))
        o.sweep(1, mode="direct")
        s = o.spins()
        for t in range(o.R):
            counts[t, int(sum(int(v) * q ** (L - 1 - i) for i, v in enumerate(s[t])))] += 1
    import itertools
    states = list(itertools.product(range(q), repeat=L))
    index = {st: n for n, st in enumerate(states)}
    E = np.array([-0.5 * c * sum(J[abs(i - j) % L] for i in range(L) for j in range(L) if i != j and st[i] == st[j])
                  for st in states])
    for t in range(o.R):
        beta = 1.0 / temps[t]
        Pbar = np.zeros((len(states), len(states)))
        for k in range(L):
            for n, st in enumerate(states):
                for x in range(q):
                    if x == st[k]:
                        continue
                    m = index[st[:k] + (x,) + st[k + 1:]]
                    p = min(1.0, math.exp(-beta * (E[m] - E[n]))) / (q - 1) / L
                    Pbar[n, m] += p
                    Pbar[n, n] += 1.0 / (q - 1) / L - p
        T = np.linalg.matrix_power(Pbar, L)
        pi = np.exp(-beta * (E - E.min()))
        pi /= pi.sum()
        np.testing.assert_allclose(pi @ T, pi, atol=1e-13)
        Tseq, _, _ = _one_sweep_kernel(L, q, J, c, beta, "metropolis")
        row0 = index[tuple(int(v) for v in s0)]

        def stat(p):
            msk = p * nsamp > 5
            return ((counts[t][msk] - nsamp * p[msk]) ** 2 / (nsamp * p[msk])).sum(), int(msk.sum()) - 1

        x2, dof = stat(T[row0])
        assert chi2.sf(x2, dof) > 1e-4, (t, x2, dof)
        x2s, dofs = stat(Tseq[row0])
        assert chi2.sf(x2s, dofs) < 1e-6, (t, x2s, dofs)


def test_random_site_chain_samples_boltzmann():
    """Random-site PT at L = 8, q = 3 samples exp(-beta H): <E> and <M> per slot
    agree with exact enumeration within 3 binned standard errors."""
    L, q, sigma, c = 8, 3, 0.5, 2
    ratios = (0.15, 0.3, 0.6)
    temps = np.array(ratios) * jtot(L, sigma)
    o = Oracle(L, q, sigma, temps, seed=777, c=c, site_order="random")
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
        for name, series in (("E", E[:, t]), ("M", M[:, t])):
            mean, se = _binned(series)
            var = ex[name + "2"][t] - ex[name][t] ** 2
            se = max(se, math.sqrt(max(var, 0.0) / n))
            assert abs(mean - ex[name][t]) < 3.0 * se + 1e-12, (t, name, mean, ex[name][t], se)
