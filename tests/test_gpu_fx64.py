"""FX64 mode (64-bit fixed-point fields, exact integer updates, FP64 decisions)
through the C ABI against the CPU oracle's FP64 chain on the same seeded
inputs: spin trajectories bit-exact (no near tie occurs at these sizes; the
oracle reports any), energies to 1e-10 relative, fields within 1e-12 Jtot of
the oracle's FP64 fields.  The fields are exact: a rebuild from the spins
reproduces them bit for bit.  Batching, checkpoints and the field residencies
give the same results as the job alone."""
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


def _temps(L, sigma, R, lo=0.05, hi=1.0):
    return workloads.geometric_ratios(R, lo, hi) * oracle.jtot(L, sigma)


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
    assert gs["near_metro"] == 0 and gs["near_exch"] == 0, what
    np.testing.assert_array_equal(gs["acc_flip"], st["acc_flip"], err_msg=what)
    np.testing.assert_array_equal(gs["acc_swap"], st["acc_swap"], err_msg=what)


def test_fx64_parity_small_job_1000_sweeps(plr):
    """L=64, q=3, sigma=0.5, R=16, seed 1: 1000 sweeps + exchanges against the
    oracle's direct-sum FP64 chain, compared every 100 steps."""
    spec = workloads.parity_job()
    temps = spec.ratios * oracle.jtot(spec.L, spec.sigma)
    g = plr.Job(spec.L, spec.q, spec.sigma, temps, spec.seed, precision="fx64")
    o = oracle.Oracle(spec.L, spec.q, spec.sigma, temps, spec.seed, fields=False)
    _compare(g, o, "initial")
    for n in range(spec.sweeps):
        g.sweep(1)
        g.exchange()
        o.sweep(1, mode="direct")
        o.exchange()
        if (n + 1) % 100 == 0:
            _compare(g, o, "step %d" % (n + 1))
    assert g.stats()["acc_flip"].sum() > 1000
    g.close()


@pytest.mark.parametrize("L,q,sigma,R,c,seed,variant", [
    (100, 7, 0.3, 5, 1, 3, "auto"),     # ragged L, pair-once
    (2, 2, 0.5, 3, 2, 4, "auto"),       # smallest chain
    (33, 16, 0.9, 1, 2, 5, "auto"),     # largest q, single slot
    (257, 4, 0.15, 9, 2, 6, "auto"),    # several site blocks + ragged tail
    (257, 4, 0.15, 9, 2, 6, "global"),  # the same with the fields in global memory
    (4096, 8, 0.2, 2, 2, 21, "auto"),   # 256 KB of fields: global memory, table in shared memory
])
def test_fx64_parity_shapes(plr, L, q, sigma, R, c, seed, variant):
    temps = _temps(L, sigma, R, 0.05, 1.0 if L < 4096 else 0.5)
    g = plr.Job(L, q, sigma, temps, seed, precision="fx64", pair_factor=c, sweep_variant=variant)
    o = oracle.Oracle(L, q, sigma, temps, seed, c=c, fields=True)
    steps = 60 if L < 4096 else 3
    for _ in range(steps):
        g.sweep(1)
        g.exchange()
        o.step(mode="field")
    _compare(g, o, "L=%d q=%d %s" % (L, q, variant))
    np.testing.assert_allclose(g.fields(), o.fields(), rtol=0, atol=1e-12 * oracle.jtot(L, sigma))
    g.close()


def test_fx64_fields_are_exact(plr):
    """After many accepted flips the fields equal, bit for bit, the integer
    direct sums from the spins (a rebuild changes nothing), and they are
    within 1e-13 Jtot of the FP64 direct sums."""
    L, q, sigma, R = 1000, 5, 0.4, 6
    g = plr.Job(L, q, sigma, _temps(L, sigma, R), 9, precision="fx64")
    for _ in range(5):
        g.sweep(20)
        g.exchange()
    assert g.stats()["acc_flip"].sum() > 10 * L
    F = g.fields()
    E = g.running_energy()
    g.fields_recompute()
    np.testing.assert_array_equal(g.fields(), F)
    np.testing.assert_allclose(g.running_energy(), E, rtol=1e-12)
    assert g.fields_error() < 1e-13
    # sum over states of h[x][i] is the same at every site (Jtot up to rounding)
    s = F.sum(axis=1)
    assert np.ptp(s) < 1e-12 * oracle.jtot(L, sigma)
    g.close()


def test_fx64_equals_fp64_on_chain_shape(plr):
    """The L=1024, q=5, sigma=0.4 chain shape, 8 of its 64 slots, 40 steps:
    FX64 and FP64 give the same spins and acceptance counts, and both follow
    the oracle."""
    spec = workloads.chains_jobs()[0]
    temps = spec.ratios[::8] * oracle.jtot(spec.L, spec.sigma)
    gx = plr.Job(spec.L, spec.q, spec.sigma, temps, spec.seed, precision="fx64")
    g64 = plr.Job(spec.L, spec.q, spec.sigma, temps, spec.seed, precision="fp64")
    o = oracle.Oracle(spec.L, spec.q, spec.sigma, temps, spec.seed)
    for _ in range(40):
        for g in (gx, g64):
            g.sweep(1)
            g.exchange()
        o.step(mode="field")
    _compare(gx, o, "fx64")
    np.testing.assert_array_equal(gx.spins(), g64.spins())
    np.testing.assert_array_equal(gx.stats()["acc_flip"], g64.stats()["acc_flip"])
    np.testing.assert_allclose(gx.fields(), g64.fields(), rtol=0, atol=1e-12 * oracle.jtot(spec.L, spec.sigma))
    gx.close()
    g64.close()


def test_fx64_batch_and_checkpoint(plr):
    """An FX64 job batched with FP64 and FP32 jobs gets exactly its results
    alone; a checkpoint taken mid-run resumes bit for bit."""
    specs = [(300, 6, 0.5, 8, 11, "fx64"), (64, 3, 0.5, 4, 12, "fp64"), (500, 4, 0.7, 5, 13, "fp32"),
             (1024, 5, 0.4, 16, 14, "fx64")]

    def make(sp):
        L, q, sigma, R, seed, prec = sp
        return plr.Job(L, q, sigma, _temps(L, sigma, R), seed, precision=prec, recompute_every=10)

    alone = []
    for sp in specs:
        j = make(sp)
        for _ in range(17):
            j.sweep(1)
            j.exchange()
        alone.append((j.spins(), j.fields(), j.running_energy()))
        j.close()
    jobs = [make(sp) for sp in specs]
    b = plr.Batch(jobs)
    b.run(17, 5)
    b.sync()
    for sp, j, (S, F, E) in zip(specs, jobs, alone):
        np.testing.assert_array_equal(j.spins(), S, err_msg=str(sp))
        np.testing.assert_array_equal(j.fields(), F, err_msg=str(sp))
        np.testing.assert_array_equal(j.running_energy(), E, err_msg=str(sp))
    b.close()
    for j in jobs:
        j.close()

    L, q, sigma, R, seed, _ = specs[0]
    a = make(specs[0])
    for _ in range(10):
        a.sweep(1)
        a.exchange()
    state = a.get_state()
    for _ in range(10):
        a.sweep(1)
        a.exchange()
    c = make(specs[0])
    c.set_state(state)
    for _ in range(10):
        c.sweep(1)
        c.exchange()
    np.testing.assert_array_equal(c.spins(), a.spins())
    np.testing.assert_array_equal(c.fields(), a.fields())
    np.testing.assert_array_equal(c.running_energy(), a.running_energy())
    assert c.counters() == a.counters() == (20, 20)
    a.close()
    c.close()


def test_fx64_full_size_chains_in_bench_configuration(plr):
    """The eight L=1024, q=5, R=64 chains (seeds 1..8) stepped as one batch, the
    bench's launch configuration (512 slots, SM placement plan), for 20 steps in
    FX64 and in FP64: identical spins and acceptance counts at full size;
    energies and magnetisations of two chains against the oracle's plain double
    sum on the GPU's configurations; the running energy against the measured
    one; FX64 fields unchanged by a rebuild."""
    specs = workloads.chains_jobs()

    def run(prec):
        jobs = [plr.Job(s.L, s.q, s.sigma, s.ratios * oracle.jtot(s.L, s.sigma), s.seed, precision=prec)
                for s in specs]
        b = plr.Batch(jobs)
        for _ in range(20):
            b.sweep(1)
            b.exchange()
        b.sync()
        return b, jobs

    bx, jx = run("fx64")
    b64, j64 = run("fp64")
    for s, a, c in zip(specs, jx, j64):
        np.testing.assert_array_equal(a.spins(), c.spins(), err_msg="seed %d" % s.seed)
        sa, sc = a.stats(), c.stats()
        np.testing.assert_array_equal(sa["acc_flip"], sc["acc_flip"])
        np.testing.assert_array_equal(sa["acc_swap"], sc["acc_swap"])
    for s, a in list(zip(specs, jx))[:2]:
        temps = s.ratios * oracle.jtot(s.L, s.sigma)
        E, M = a.measure()
        o = oracle.Oracle(s.L, s.q, s.sigma, temps, s.seed, fields=False)
        o.set_spins(a.spins())
        np.testing.assert_allclose(E, o.energy(), rtol=1e-10)
        np.testing.assert_allclose(M, o.magnetisation(), rtol=0, atol=1e-14)
        np.testing.assert_allclose(a.running_energy(), E, rtol=1e-10)
    F = jx[0].fields()
    jx[0].fields_recompute()
    np.testing.assert_array_equal(jx[0].fields(), F)
    for b in (bx, b64):
        b.close()
    for j in jx + j64:
        j.close()


@pytest.mark.parametrize("L,q,variant", [(64, 3, "direct"), (64, 3, "registers7"), (4096, 8, "registers"),
                                         (1200, 6, "registers"), (500, 9, "registers3")])
def test_fx64_rejects_unsupported_variants(plr, L, q, variant):
    """No direct sweep in FX64 mode, no FX64 register configuration 7 or 8,
    and none that does not hold the chain."""
    from paper_1308_5426_gb300 import _lib
    with pytest.raises(_lib.PottsError) as ei:
        plr.Job(L, q, 0.5, _temps(L, 0.5, 2), 1, precision="fx64", sweep_variant=variant)
    assert ei.value.code == _lib.EINVAL


@pytest.mark.parametrize("L,q,sigma,R,cfg", [
    (200, 16, 0.6, 5, 1), (33, 5, 0.4, 3, 1), (448, 9, 0.3, 4, 2), (300, 2, 0.8, 6, 2),
    (1024, 5, 0.4, 12, 3), (1000, 8, 0.2, 5, 3), (1120, 7, 0.5, 4, 4), (999, 3, 0.9, 5, 4),
    (2400, 5, 0.4, 3, 5), (1500, 2, 0.3, 4, 5), (4320, 3, 0.5, 2, 6), (3001, 2, 0.7, 3, 6),
])
def test_fx64_register_configurations_equal_the_memory_kernel(plr, L, q, sigma, R, cfg):
    """Every FX64 register configuration (64-bit integer fields in registers,
    a decision warp taking the FP64 rule) against the shared/global-memory
    FX64 kernel: identical spins, fields, energies (the exact 128-bit sum) and
    counters after sweeps, exchanges and multi-sweep launches."""
    temps = _temps(L, sigma, R)
    a = plr.Job(L, q, sigma, temps, 31, precision="fx64", sweep_variant="memory")
    b = plr.Job(L, q, sigma, temps, 31, precision="fx64", sweep_variant="registers%d" % cfg)
    assert b.sweep_info()["kernel"] == "registers" and b.sweep_info()["register_config"] == cfg
    for _ in range(8):
        for j in (a, b):
            j.sweep(1)
            j.exchange()
    for j in (a, b):
        j.sweep(3)
    np.testing.assert_array_equal(a.spins(), b.spins())
    np.testing.assert_array_equal(a.fields(), b.fields())
    np.testing.assert_array_equal(a.running_energy(), b.running_energy())
    sa, sb = a.stats(), b.stats()
    np.testing.assert_array_equal(sa["acc_flip"], sb["acc_flip"])
    np.testing.assert_array_equal(sa["acc_swap"], sb["acc_swap"])
    assert sa["near_metro"] == sb["near_metro"]
    a.close()
    b.close()
