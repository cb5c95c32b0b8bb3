"""GPU parity: the CUDA path through the C ABI against the CPU oracle on the
same seeded inputs.  FP64 mode: spin trajectories bit-exact (no near tie may
occur at these sizes; the oracle reports any), energies to 1e-10 relative."""
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


def _pair(plr, L, q, sigma, ratios, seed, c=2, precision="fp64", K=100, fields=True):
    temps = np.asarray(ratios) * oracle.jtot(L, sigma)
    g = plr.Job(L, q, sigma, temps, seed, precision=precision, recompute_every=K, pair_factor=c)
    o = oracle.Oracle(L, q, sigma, temps, seed, c=c, fields=fields)
    return g, o


def _compare(g, o, what=""):
    st = o.stats()
    assert st["near_metro"].sum() == 0 and st["near_exch"] == 0, "oracle saw a near tie; pick other seeds"
    np.testing.assert_array_equal(g.spins(), o.spins(), err_msg=what)
    E, M = g.measure()
    Eo = o.energy()
    np.testing.assert_allclose(E, Eo, rtol=1e-10, atol=1e-10 * np.abs(Eo).max(), err_msg=what)
    np.testing.assert_allclose(M, o.magnetisation(), rtol=0, atol=1e-14, err_msg=what)
    np.testing.assert_allclose(g.running_energy(), o.running_energy(), rtol=1e-10,
                               atol=1e-10 * np.abs(Eo).max(), err_msg=what)
    gs = g.stats()
    np.testing.assert_array_equal(gs["acc_flip"], st["acc_flip"], err_msg=what)
    np.testing.assert_array_equal(gs["acc_swap"], st["acc_swap"], err_msg=what)


def test_initial_state(plr):
    spec = workloads.parity_job()
    g, o = _pair(plr, spec.L, spec.q, spec.sigma, spec.ratios, spec.seed)
    _compare(g, o, "initial")
    np.testing.assert_allclose(g.fields(), o.fields(), rtol=0, atol=1e-13 * oracle.jtot(spec.L, spec.sigma))


def test_parity_small_job_1000_sweeps(plr):
    """L=64, q=3, sigma=0.5, R=16, T/Jtot geometric in [0.05, 1], seed 1, sweep +
    exchange 1000 times, compared every 100 steps (oracle in direct-sum mode)."""
    spec = workloads.parity_job()
    g, o = _pair(plr, spec.L, spec.q, spec.sigma, spec.ratios, spec.seed, fields=False)
    for n in range(spec.sweeps):
        g.sweep(1)
        g.exchange()
        o.sweep(1, mode="direct")
        o.exchange()
        if (n + 1) % 100 == 0:
            _compare(g, o, "step %d" % (n + 1))
    assert g.stats()["acc_flip"].sum() > 1000  # the chain moves


@pytest.mark.parametrize("L,q,sigma,R,c,seed", [
    (100, 7, 0.3, 5, 1, 3),      # ragged L (not a multiple of 8 or 32), pair-once
    (2, 2, 0.5, 3, 2, 4),        # smallest chain
    (33, 16, 0.9, 1, 2, 5),      # largest q, single slot (no exchange pairs)
    (257, 4, 0.15, 9, 2, 6),     # several site blocks + ragged tail, odd R
])
def test_parity_shapes(plr, L, q, sigma, R, c, seed):
    ratios = workloads.geometric_ratios(R, 0.05, 1.0)
    g, o = _pair(plr, L, q, sigma, ratios, seed, c=c)
    for n in range(60):
        g.sweep(1)
        g.exchange()
        o.step(mode="field")
    _compare(g, o, "L=%d q=%d" % (L, q))
    np.testing.assert_allclose(g.fields(), o.fields(), rtol=0, atol=1e-12 * oracle.jtot(L, sigma))


@pytest.mark.parametrize("L,q,sigma,R,sweeps", [
    (4096, 8, 0.2, 2, 3),    # FP64 fields (256 KB) stay in global memory, table in shared memory
    (9000, 16, 0.7, 1, 1),   # neither fields nor table in shared memory, ragged L
])
def test_parity_fields_in_global_memory(plr, L, q, sigma, R, sweeps):
    ratios = workloads.geometric_ratios(R, 0.05, 0.5)
    g, o = _pair(plr, L, q, sigma, ratios, 21)
    for _ in range(sweeps):
        g.sweep(1)
        g.exchange()
        o.step(mode="field")
    _compare(g, o, "global-memory fields L=%d" % L)
    np.testing.assert_allclose(g.fields(), o.fields(), rtol=0, atol=1e-12 * oracle.jtot(L, sigma))


def test_parity_multi_sweep_launch(plr):
    """sweep(n) with n > 1 in one launch equals n single sweeps."""
    L, q, sigma, R = 96, 5, 0.4, 4
    ratios = workloads.geometric_ratios(R, 0.05, 1.0)
    g, o = _pair(plr, L, q, sigma, ratios, 8)
    for _ in range(5):
        g.sweep(7)
        g.exchange()
        o.sweep(7)
        o.exchange()
    _compare(g, o, "multi-sweep")


def test_parity_chain_shape_subset(plr):
    """The L=1024, q=5, sigma=0.4 chain shape with 8 of its 64 slots, 30 steps."""
    spec = workloads.chains_jobs()[0]
    ratios = spec.ratios[::8]
    g, o = _pair(plr, spec.L, spec.q, spec.sigma, ratios, spec.seed)
    for _ in range(30):
        g.sweep(1)
        g.exchange()
        o.step(mode="field")
    _compare(g, o, "L=1024 subset")


def test_full_size_chains_sampled(plr):
    """Eight L=1024, q=5, R=64 chains (seeds 1..8) at full size for 20 steps:
    energies and magnetisations of every slot against the oracle's plain
    double sum evaluated on the GPU's configurations (sampled outputs), and the
    running energy against the measured one."""
    for spec in workloads.chains_jobs()[:8]:
        temps = spec.ratios * oracle.jtot(spec.L, spec.sigma)
        g = plr.Job(spec.L, spec.q, spec.sigma, temps, spec.seed)
        for _ in range(20):
            g.sweep(1)
            g.exchange()
        E, M = g.measure()
        S = g.spins()
        o = oracle.Oracle(spec.L, spec.q, spec.sigma, temps, spec.seed, fields=False)
        o.set_spins(S)
        Eo = o.energy()
        np.testing.assert_allclose(E, Eo, rtol=1e-10)
        np.testing.assert_allclose(M, o.magnetisation(), atol=1e-14)
        np.testing.assert_allclose(g.running_energy(), E, rtol=1e-10)
        assert S.max() < spec.q
        g.close()


def test_checkpoint_resume_bit_exact(plr):
    L, q, sigma, R = 128, 4, 0.5, 6
    ratios = workloads.geometric_ratios(R, 0.05, 1.0)
    temps = ratios * oracle.jtot(L, sigma)
    a = plr.Job(L, q, sigma, temps, 11)
    for _ in range(10):
        a.sweep(1)
        a.exchange()
    st = a.get_state()
    for _ in range(15):
        a.sweep(1)
        a.exchange()
    b = plr.Job(L, q, sigma, temps, 11)
    b.set_state(st)
    for _ in range(15):
        b.sweep(1)
        b.exchange()
    np.testing.assert_array_equal(a.spins(), b.spins())
    np.testing.assert_array_equal(a.running_energy(), b.running_energy())
    np.testing.assert_array_equal(a.fields(), b.fields())
    assert a.counters() == b.counters()
    with pytest.raises(plr.PottsError):
        c = plr.Job(L + 32, q, sigma, temps, 11)
        c.set_state(st)


def test_zero_and_infinite_temperature_limits(plr):
    """beta -> 0: every proposal is accepted; beta -> infinity: only dE <= 0
    moves are (a greedy quench).  Both degenerate chains equal the oracle's."""
    L, q, sigma = 64, 3, 0.5
    hot = plr.Job(L, q, sigma, np.full(3, 1e300), 9)
    oh = oracle.Oracle(L, q, sigma, np.full(3, 1e300), 9)
    hot.sweep(3)
    oh.sweep(3)
    assert hot.stats()["acc_flip"].tolist() == [3 * L] * 3
    np.testing.assert_array_equal(hot.spins(), oh.spins())
    cold = plr.Job(L, q, sigma, np.full(2, 1e-9), 5)
    oc = oracle.Oracle(L, q, sigma, np.full(2, 1e-9), 5)
    for _ in range(10):
        cold.sweep(1)
        cold.exchange()
        oc.step()
    np.testing.assert_array_equal(cold.spins(), oc.spins())
    E, _ = cold.measure()
    np.testing.assert_allclose(E, oc.energy(), rtol=1e-10)


@pytest.mark.parametrize("L,q,sigma,R,c,seed,steps", [
    (64, 3, 0.5, 16, 2, 1, 300),   # the small parity job
    (257, 4, 0.15, 6, 1, 6, 40),   # ragged tail, pair-once
    (33, 16, 0.9, 2, 2, 5, 60),    # largest q
    (1024, 5, 0.4, 8, 2, 3, 8),    # the chain shape
])
def test_parity_direct_sweep(plr, L, q, sigma, R, c, seed, steps):
    """The direct sweep (the paper's scheme: every proposal sums its O(L)
    interaction, no fields) follows the oracle's direct mode bit for bit;
    fields read back from such a job are rebuilt exactly."""
    temps = workloads.geometric_ratios(R, 0.05, 1.0) * oracle.jtot(L, sigma)
    g = plr.Job(L, q, sigma, temps, seed, precision="fp64", pair_factor=c, sweep_variant="direct")
    o = oracle.Oracle(L, q, sigma, temps, seed, c=c)
    for _ in range(steps):
        g.sweep(1)
        g.exchange()
        o.sweep(1, mode="direct")
        o.exchange()
    _compare(g, o, "direct L=%d" % L)
    np.testing.assert_allclose(g.fields(), o.fields(), rtol=0, atol=1e-12 * oracle.jtot(L, sigma))
    with pytest.raises(plr.PottsError):
        plr.Job(L, q, sigma, temps, seed, precision="fp32", sweep_variant="direct")


@pytest.mark.parametrize("L,q,sigma,R,seed,steps", [
    (64, 3, 0.5, 16, 1, 200),
    (257, 4, 0.15, 6, 6, 30),
    (1000, 5, 0.4, 4, 3, 6),
])
def test_parity_random_site_order(plr, L, q, sigma, R, seed, steps):
    """Random site order (attempt m of a sweep at a Philox-drawn site) on the
    direct sweep follows the oracle's random-site chain bit for bit."""
    temps = workloads.geometric_ratios(R, 0.05, 1.0) * oracle.jtot(L, sigma)
    g = plr.Job(L, q, sigma, temps, seed, precision="fp64", site_order="random")
    o = oracle.Oracle(L, q, sigma, temps, seed, site_order="random")
    for _ in range(steps):
        g.sweep(1)
        g.exchange()
        o.sweep(1, mode="direct")
        o.exchange()
    _compare(g, o, "random sites L=%d" % L)
    for bad in (dict(precision="fp32"), dict(precision="fp64", sweep_variant="memory")):
        with pytest.raises(plr.PottsError):
            plr.Job(L, q, sigma, temps, seed, site_order="random", **bad)
