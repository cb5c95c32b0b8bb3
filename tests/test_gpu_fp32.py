"""FP32 mode: fields in FP32, re-anchored every K sweeps by the split-BF16
tensor-core rebuild H = C . onehot(S).  Checked against FP64: the rebuild
error and the field drift stay below 1e-5 of Jtot (drift = max over slots,
states and sites of |h32 - h64| / Jtot, h64 the FP64 direct rebuild of the
same spins), and FP32 chains sample the same <E> and <M> as FP64 chains
within 3 binned standard errors."""
import math

import numpy as np
import pytest

import oracle
from paper_1308_5426_gb300 import workloads

pytestmark = pytest.mark.gpu

DRIFT_BOUND = 1e-5


@pytest.fixture(scope="module")
def plr():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1308_5426_gb300
    return paper_1308_5426_gb300


@pytest.mark.parametrize("L,q,R,sigma", [
    (64, 3, 4, 0.5), (200, 5, 7, 0.3), (1000, 16, 9, 0.9), (1024, 5, 64, 0.4),
    (4096, 8, 128, 0.2), (16384, 8, 64, 0.1), (300, 2, 3, 1.5),
])
def test_tensor_core_rebuild_accuracy(plr, L, q, R, sigma):
    temps = workloads.geometric_ratios(R, 0.05, 1.0) * oracle.jtot(L, sigma)
    j = plr.Job(L, q, sigma, temps, 3, precision="fp32", recompute_every=0)
    j.sweep(2)
    j.fields_recompute()
    err = j.fields_error()
    assert err < DRIFT_BOUND, err
    # the rebuilt fields satisfy sum_x h[x][i] = Jtot within the per-field bound
    h = j.fields()
    np.testing.assert_allclose(h.sum(axis=1), oracle.jtot(L, sigma), rtol=DRIFT_BOUND)
    # re-anchored running energy equals the measured one
    E, _ = j.measure()
    np.testing.assert_allclose(j.running_energy(), E, rtol=1e-12)


@pytest.mark.parametrize("L,q,R,sigma", [(4096, 8, 128, 0.2), (16384, 5, 64, 0.4), (1024, 5, 64, 0.4)])
def test_rebuild_split_two_and_three_parts(plr, L, q, R, sigma):
    """The split of J* into BF16 parts: three (hi + mid + lo) and two (hi +
    mid) both rebuild within the 1e-5 Jtot bound; three parts are measured
    several times more accurate (on GB300: 2e-8..1.1e-7 against 2.8e-7..9.6e-7
    Jtot), which is why explicit rebuilds and slow schedules use them."""
    temps = workloads.geometric_ratios(R, 0.05, 1.0) * oracle.jtot(L, sigma)
    err = {}
    for parts in (3, 2):
        j = plr.Job(L, q, sigma, temps, 3, precision="fp32", recompute_every=0)
        j.sweep(3)
        j.set_rebuild_split(parts)
        j.fields_recompute()
        err[parts] = j.fields_error()
        j.close()
    print("L=%d q=%d: rebuild error, 3 parts %.3e, 2 parts %.3e Jtot" % (L, q, err[3], err[2]))
    assert err[3] < 2e-7 and err[2] < 1e-6
    assert err[3] < err[2]


def test_automatic_split_and_energy_anchor_on_fast_schedules(plr):
    """With rebuilds every sweep (K = 1) the automatic split is the two-part
    one (identical to asking for it, unlike three parts), and the running
    energy, re-anchored from the spins every 8 sweeps, carries the FP32
    fields' error in between (measured about 3e-5 Jtot per sweep; bounded here
    by 1e-3 Jtot); an explicit rebuild re-anchors it at once."""
    L, q, sigma, R = 4096, 5, 0.4, 8
    temps = workloads.geometric_ratios(R, 0.05, 1.0) * oracle.jtot(L, sigma)
    jobs = {}
    for name, parts in (("auto", None), ("two", 2), ("three", 3)):
        j = plr.Job(L, q, sigma, temps, 11, precision="fp32", recompute_every=1)
        if parts is not None:
            j.set_rebuild_split(parts)
        for _ in range(13):
            j.sweep(1)
            j.exchange()
        jobs[name] = j
    np.testing.assert_array_equal(jobs["auto"].fields(), jobs["two"].fields())
    np.testing.assert_array_equal(jobs["auto"].spins(), jobs["two"].spins())
    assert not np.array_equal(jobs["auto"].fields(), jobs["three"].fields())
    j = jobs["auto"]
    assert j.fields_error() < DRIFT_BOUND
    E, _ = j.measure()
    np.testing.assert_allclose(j.running_energy(), E, rtol=0, atol=1e-3 * oracle.jtot(L, sigma))
    j.fields_recompute()
    E, _ = j.measure()
    np.testing.assert_allclose(j.running_energy(), E, rtol=1e-12)
    for j in jobs.values():
        j.close()


def test_rebuild_schedule_is_reported(plr):
    """potts_lr_rebuild_info: the adaptive interval, the rebuilds done and the
    last measured drift of an FP32 job with K = 100."""
    L, q, sigma, R = 4096, 8, 0.5, 16
    temps = workloads.geometric_ratios(R, 0.05, 1.0) * oracle.jtot(L, sigma)
    j = plr.Job(L, q, sigma, temps, 5, precision="fp32", recompute_every=100)
    assert j.rebuild_info()["rebuilds"] == 0
    for _ in range(120):
        j.sweep(1)
        j.exchange()
    info = j.rebuild_info()
    print("L=%d q=%d after 120 sweeps: %s" % (L, q, info))
    assert info["rebuilds"] >= 2 and 1 <= info["interval"] <= 100
    assert 0.0 < info["last_drift"] < 1e-5
    g = plr.Job(L, q, sigma, temps, 5, precision="fp64")
    g.sweep(2)
    assert g.rebuild_info() == {"interval": 0, "rebuilds": 0, "last_drift": 0.0}
    with pytest.raises(plr.PottsError):
        g.set_rebuild_split(2)
    j.close()
    g.close()


def test_tensor_core_rebuild_small_matches_oracle_fields(plr):
    """Rebuilt FP32 fields against the oracle's FP64 fields of the same spins."""
    L, q, R, sigma = 96, 4, 3, 0.6
    temps = workloads.geometric_ratios(R, 0.05, 1.0) * oracle.jtot(L, sigma)
    j = plr.Job(L, q, sigma, temps, 5, precision="fp32", recompute_every=0)
    j.sweep(3)
    j.fields_recompute()
    o = oracle.Oracle(L, q, sigma, temps, 5)
    o.set_spins(j.spins())
    np.testing.assert_allclose(j.fields(), o.fields(), rtol=0, atol=2e-6 * oracle.jtot(L, sigma))


@pytest.mark.parametrize("L,q,sigma,lo,hi,R,seed,sweeps,every", [
    (4096, 8, 0.2, 0.02, 0.5, 16, 1, 160, 10),   # the precision workload's shape, 16 of its slots
    (16384, 3, 0.817, 0.05, 1.0, 8, 25, 40, 4),  # the hardest serving shape: long chain, few states
    (8192, 3, 0.659, 0.05, 1.0, 8, 10, 60, 5),
])
def test_drift_stays_below_bound(plr, L, q, sigma, lo, hi, R, seed, sweeps, every):
    """With recompute_every = 100 the adaptive schedule keeps the FP32 field
    drift below 1e-5 Jtot at every check, not only right after a rebuild."""
    temps = workloads.geometric_ratios(R, lo, hi) * oracle.jtot(L, sigma)
    j = plr.Job(L, q, sigma, temps, seed, precision="fp32", recompute_every=100)
    worst = 0.0
    for n in range(sweeps):
        j.sweep(1)
        j.exchange()
        if (n + 1) % every == 0:
            worst = max(worst, j.fields_error())
    print("L=%d q=%d: worst drift %.3e over %d sweeps" % (L, q, worst, sweeps))
    assert worst < DRIFT_BOUND, worst


def _binned(x, nbins=20):
    x = np.asarray(x)
    b = x[: (x.size // nbins) * nbins].reshape(nbins, -1).mean(axis=1)
    return b.mean(), b.std(ddof=1) / math.sqrt(nbins)


def test_fp32_and_fp64_sample_the_same_observables(plr):
    """Same seeds, same call sequence: <E>/L and <M> per temperature from an
    FP32 chain and an FP64 chain agree within 3 binned standard errors
    (combined), after equilibration.  L=256, q=3, sigma=0.5, R=8."""
    L, q, sigma, R = 256, 3, 0.5, 8
    temps = workloads.geometric_ratios(R, 0.05, 1.0) * oracle.jtot(L, sigma)
    res = {}
    for prec in ("fp32", "fp64"):
        j = plr.Job(L, q, sigma, temps, 17, precision=prec, recompute_every=100)
        for _ in range(300):
            j.sweep(1)
            j.exchange()
        Es, Ms = [], []
        for _ in range(400):
            j.sweep(5)
            j.exchange()
            E, M = j.measure()
            Es.append(E / L)
            Ms.append(M)
        res[prec] = (np.array(Es), np.array(Ms))
    for k, name in ((0, "E"), (1, "M")):
        for t in range(R):
            m32, s32 = _binned(res["fp32"][k][:, t])
            m64, s64 = _binned(res["fp64"][k][:, t])
            se = math.hypot(s32, s64)
            assert abs(m32 - m64) < 3 * se + 1e-9, (name, t, m32, m64, se)


@pytest.mark.parametrize("L,q,sigma,R", [
    (65, 4, 0.5, 4), (96, 3, 0.6, 3), (200, 3, 0.5, 4), (256, 16, 0.3, 3), (500, 5, 0.7, 5), (500, 11, 0.7, 3),
    (1000, 16, 0.4, 3), (1024, 5, 0.4, 8), (1536, 7, 0.5, 3), (2048, 8, 0.6, 3), (1999, 2, 0.2, 4),
    (4096, 8, 0.2, 3), (4224, 3, 0.3, 2), (3000, 6, 0.9, 2), (6000, 5, 0.4, 2), (10000, 3, 0.2, 2),
    (16000, 2, 0.6, 2), (2000, 10, 0.5, 3), (2400, 9, 0.3, 2),
])
def test_register_path_equals_memory_path(plr, L, q, sigma, R):
    """The register-resident FP32 sweep and the shared/global-memory FP32 sweep
    run the same arithmetic: spins, fields, energies and counters agree bit for
    bit after sweeps, exchanges and tensor-core rebuilds."""
    temps = workloads.geometric_ratios(R, 0.05, 1.0) * oracle.jtot(L, sigma)
    a = plr.Job(L, q, sigma, temps, 9, precision="fp32", recompute_every=6, sweep_variant="memory")
    b = plr.Job(L, q, sigma, temps, 9, precision="fp32", recompute_every=6, sweep_variant="registers")
    for _ in range(15):
        a.sweep(1)
        a.exchange()
        b.sweep(1)
        b.exchange()
    a.sweep(3)
    b.sweep(3)
    np.testing.assert_array_equal(a.spins(), b.spins())
    np.testing.assert_array_equal(a.fields(), b.fields())
    np.testing.assert_array_equal(a.running_energy(), b.running_energy())
    np.testing.assert_array_equal(a.stats()["acc_flip"], b.stats()["acc_flip"])


@pytest.mark.parametrize("L,q", [(8192, 10), (4400, 6), (2048, 11), (2500, 9), (8000, 4), (13000, 3), (17000, 2)])
def test_register_path_rejects_unsupported_shapes(plr, L, q):
    temps = np.linspace(1.0, 2.0, 2)
    with pytest.raises(plr.PottsError):
        plr.Job(L, q, 0.5, temps, 1, precision="fp32", sweep_variant="registers")


@pytest.mark.parametrize("precision,L,q,sigma,R", [
    ("fp32", 2048, 5, 0.4, 3), ("fp32", 700, 11, 0.6, 3), ("fp32", 1000, 3, 0.3, 4),
    ("fp64", 1024, 5, 0.4, 3), ("fp64", 333, 9, 0.7, 3),
])
def test_shared_and_global_field_residency_agree(plr, precision, L, q, sigma, R):
    """Fields in shared memory and in global memory (and, in FP32 mode, in
    registers) run the same arithmetic: identical spins, fields, energies."""
    temps = workloads.geometric_ratios(R, 0.05, 1.0) * oracle.jtot(L, sigma)
    variants = ["memory", "global"] + (["registers"] if precision == "fp32" and q <= 8 else [])
    jobs = [plr.Job(L, q, sigma, temps, 17, precision=precision, recompute_every=6, sweep_variant=v)
            for v in variants]
    for _ in range(12):
        for j in jobs:
            j.sweep(1)
            j.exchange()
    for j in jobs[1:]:
        np.testing.assert_array_equal(jobs[0].spins(), j.spins())
        np.testing.assert_array_equal(jobs[0].fields(), j.fields())
        np.testing.assert_array_equal(jobs[0].running_energy(), j.running_energy())


@pytest.mark.parametrize("precision,L,q,sigma,R,rounds", [
    ("fp32", 2048, 5, 0.4, 3, 12),    # asked for explicitly: two CTAs, 32 blocks each
    ("fp32", 10000, 7, 0.5, 3, 6),    # automatic, two CTAs, ragged last block
    ("fp32", 16384, 12, 0.6, 2, 4),   # four CTAs
    ("fp32", 24000, 16, 0.3, 2, 2),   # eight CTAs
    ("fp64", 2048, 5, 0.4, 3, 10),    # FP64 fields: asked for, two CTAs
    ("fp64", 4096, 8, 0.2, 3, 4),     # the precision shape: two CTAs
    ("fp64", 10000, 7, 0.5, 2, 3),    # four CTAs, ragged last block
    ("fp64", 16384, 8, 0.3, 2, 2),    # eight CTAs
    ("fx64", 4096, 8, 0.2, 3, 4),     # FX64 fields: two CTAs
    ("fx64", 9000, 11, 0.6, 2, 3),    # eight CTAs, ragged
    ("fx64", 16384, 5, 0.4, 2, 2),    # four CTAs
])
def test_cluster_sweep_equals_global_sweep(plr, precision, L, q, sigma, R, rounds):
    """A slot's fields spread over the shared memory of a CTA cluster run the
    same arithmetic as the single-CTA sweep with the fields in global memory:
    spins, fields, running energies and counters agree bit for bit after
    sweeps, exchanges and (FP32) tensor-core rebuilds -- in FP32, FP64 (the
    energy summed in the single-CTA kernel's order) and FX64 (exact)."""
    temps = workloads.geometric_ratios(R, 0.05, 1.0) * oracle.jtot(L, sigma)
    a = plr.Job(L, q, sigma, temps, 23, precision=precision, recompute_every=3, sweep_variant="global")
    b = plr.Job(L, q, sigma, temps, 23, precision=precision, recompute_every=3, sweep_variant="cluster")
    assert b.sweep_info()["kernel"] == "cluster"
    for _ in range(rounds):
        for j in (a, b):
            j.sweep(1)
            j.exchange()
    a.sweep(2)
    b.sweep(2)
    np.testing.assert_array_equal(a.spins(), b.spins())
    np.testing.assert_array_equal(a.fields(), b.fields())
    np.testing.assert_array_equal(a.running_energy(), b.running_energy())
    np.testing.assert_array_equal(a.stats()["acc_flip"], b.stats()["acc_flip"])
    a.close()
    b.close()


def _spread_cluster(cmin, R, L):
    import torch
    nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    c = cmin
    while c < 8 and R * 2 * c <= 4 * nsm and (2 * c) ** 2 * 128 <= L:
        c *= 2
    return c


@pytest.mark.parametrize("precision,L,q,sigma,R,rounds", [
    ("fp64", 4096, 8, 0.2, 128, 3),   # the precision shape: 2 CTAs needed, 4 taken on 152 SMs
    ("fx64", 4096, 8, 0.2, 3, 4),     # few slots: 4 CTAs (8 would keep under 128 C sites each)
    ("fp64", 10000, 7, 0.5, 2, 2),    # 4 CTAs needed, 8 taken; ragged last block
    ("fp64", 4096, 5, 0.85, 64, 2),   # 160 KB of fields fit one CTA: a cluster all the same, 4 CTAs
])
def test_automatic_cluster_spreads_8byte_fields(plr, precision, L, q, sigma, R, rounds):
    """Chosen automatically, FP64 and FX64 fields of more than 64 KB take a
    cluster while the job's smallest clusters fit the GPU at once -- the
    largest of 2, 4 or 8 CTAs, no smaller than their shares need, whose CTAs
    still fit four per SM and hold at least 128 C sites each -- so that a hot
    slot's updates spread over more SMs; asked for explicitly, the smallest.
    Spins, fields, energies and counters equal the global-memory sweep's bit
    for bit."""
    temps = workloads.geometric_ratios(R, 0.05, 1.0) * oracle.jtot(L, sigma)
    a = plr.Job(L, q, sigma, temps, 31, precision=precision, sweep_variant="global")
    b = plr.Job(L, q, sigma, temps, 31, precision=precision)
    c = plr.Job(L, q, sigma, temps, 31, precision=precision, sweep_variant="cluster")
    cmin = c.sweep_info()["cluster"]
    c.close()
    info = b.sweep_info()
    assert info["kernel"] == "cluster"
    assert info["cluster"] == _spread_cluster(cmin, R, L) and info["cluster"] > cmin
    for _ in range(rounds):
        for j in (a, b):
            j.sweep(1)
            j.exchange()
    a.sweep(2)
    b.sweep(2)
    np.testing.assert_array_equal(a.spins(), b.spins())
    np.testing.assert_array_equal(a.fields(), b.fields())
    np.testing.assert_array_equal(a.running_energy(), b.running_energy())
    np.testing.assert_array_equal(a.stats()["acc_flip"], b.stats()["acc_flip"])
    a.close()
    b.close()


@pytest.mark.parametrize("precision,L,q,sigma,R,rounds", [
    ("fp32", 2048, 5, 0.4, 3, 8),     # two CTAs, ragged use of the second
    ("fp32", 8640, 8, 0.5, 2, 4),     # two CTAs, full
    ("fp32", 10001, 3, 0.3, 2, 3),    # four CTAs, ragged last block
    ("fp32", 16384, 5, 0.4, 2, 2),    # four CTAs (the long serving shape)
    ("fp32", 20000, 8, 0.6, 2, 2),    # eight CTAs, the last one part empty
    ("fp32", 4000, 10, 0.5, 2, 4),    # q = 9..12 (five sites per thread): two CTAs
    ("fp32", 9000, 12, 0.4, 2, 3),    # four CTAs, ragged last block
    ("fp32", 16384, 9, 0.7, 2, 2),    # eight CTAs
    ("fx64", 1000, 7, 0.5, 3, 8),     # FX64: two CTAs
    ("fx64", 9000, 5, 0.4, 2, 3),     # four CTAs
    ("fx64", 16384, 3, 0.3, 2, 2),    # eight CTAs
])
def test_register_cluster_sweep_equals_global_sweep(plr, precision, L, q, sigma, R, rounds):
    """A slot's fields held in the registers of a CTA cluster (flips sent to
    every CTA through distributed shared memory) run the same arithmetic as the
    single-CTA sweep with the fields in global memory: spins, fields, energies
    and counters agree bit for bit, across sweeps, exchanges, multi-sweep
    launches and (FP32) tensor-core rebuilds."""
    temps = workloads.geometric_ratios(R, 0.05, 1.0) * oracle.jtot(L, sigma)
    a = plr.Job(L, q, sigma, temps, 29, precision=precision, recompute_every=3, sweep_variant="global")
    b = plr.Job(L, q, sigma, temps, 29, precision=precision, recompute_every=3, sweep_variant="rcluster")
    assert b.sweep_info()["kernel"] == "register_cluster"
    for _ in range(rounds):
        for j in (a, b):
            j.sweep(1)
            j.exchange()
    for j in (a, b):
        j.sweep(2)
    np.testing.assert_array_equal(a.spins(), b.spins())
    np.testing.assert_array_equal(a.fields(), b.fields())
    np.testing.assert_array_equal(a.running_energy(), b.running_energy())
    np.testing.assert_array_equal(a.stats()["acc_flip"], b.stats()["acc_flip"])
    a.close()
    b.close()


@pytest.mark.parametrize("precision,L,q", [("fp32", 65536, 16), ("fp64", 32768, 16), ("fx64", 65536, 4)])
def test_cluster_sweep_rejects_oversize(plr, precision, L, q):
    """Fields beyond eight CTAs' shared memory (4 MB of FP32, 4 MB and 2 MB of
    8-byte words per slot) are refused."""
    temps = np.linspace(1.0, 2.0, 2)
    with pytest.raises(plr.PottsError):
        plr.Job(L, q, 0.5, temps, 1, precision=precision, sweep_variant="cluster")
