"""The sweep-shape tuner: candidate lists and variant codes (CPU), tuning and
bit-identical results of every register configuration (GPU)."""
import numpy as np
import pytest

import oracle
from paper_1308_5426_gb300 import SWEEP_VARIANTS, sweep_variant_code, workloads
from paper_1308_5426_gb300.tune import candidates


def test_variant_codes():
    assert [sweep_variant_code(v) for v in ("auto", "memory", "registers", "global", "direct", "cluster")] == [
        0, 1, 2, 3, 4, 5]
    assert [sweep_variant_code("registers%d" % c) for c in range(1, 9)] == list(range(17, 25))
    for bad in ("registers0", "registers9", "fast", 5):
        with pytest.raises(ValueError):
            sweep_variant_code(bad)
    assert len(SWEEP_VARIANTS) == 15


def test_candidates():
    assert candidates(1000, 5, "fp64") == ["auto", "memory", "global", "cluster"]
    c = candidates(1000, 5, "fp32")
    assert c[:5] == ["auto", "memory", "global", "cluster", "rcluster"]
    assert c[5:] == ["registers%d" % k for k in range(1, 9)]
    assert candidates(1000, 5, "fx64") == ["auto", "memory", "global", "cluster", "rcluster"] + [
        "registers%d" % k for k in range(1, 7)]


@pytest.fixture(scope="module")
def plr():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1308_5426_gb300
    return paper_1308_5426_gb300


@pytest.mark.gpu
def test_every_register_configuration_gives_the_same_trajectory(plr):
    """L = 200, q = 2 fits all eight register configurations: each, and the
    shared- and global-memory kernels, give identical spins, fields, energies;
    configurations that cannot hold a shape are refused."""
    L, q, sigma, R = 200, 2, 0.5, 4
    temps = workloads.geometric_ratios(R, 0.05, 1.0) * oracle.jtot(L, sigma)
    names = ["memory", "global"] + ["registers%d" % c for c in range(1, 9)]
    jobs = [plr.Job(L, q, sigma, temps, 5, precision="fp32", recompute_every=4, sweep_variant=v) for v in names]
    for _ in range(9):
        for j in jobs:
            j.sweep(1)
            j.exchange()
    for name, j in zip(names[1:], jobs[1:]):
        np.testing.assert_array_equal(jobs[0].spins(), j.spins(), err_msg=name)
        np.testing.assert_array_equal(jobs[0].fields(), j.fields(), err_msg=name)
        np.testing.assert_array_equal(jobs[0].running_energy(), j.running_energy(), err_msg=name)
    with pytest.raises(plr.PottsError):
        plr.Job(2000, 5, sigma, temps, 5, precision="fp32", sweep_variant="registers1")
    with pytest.raises(plr.PottsError):
        plr.Job(200, 3, sigma, temps, 5, precision="fp32", sweep_variant="registers8")
    with pytest.raises(plr.PottsError):
        plr.Job(200, 2, sigma, temps, 5, precision="fp64", sweep_variant="registers3")


@pytest.mark.gpu
def test_tuner_picks_a_valid_fastest_variant(plr, tmp_path):
    from paper_1308_5426_gb300 import tune
    f = str(tmp_path / "tune.json")
    best, ms = tune.tune(1024, 5, sigma=0.4, precision="fp32", R=32, sweeps=2, warm=1, cache_file=f)
    assert best in ms and ms[best] == min(ms.values())
    assert {"memory", "global", "registers3"} <= set(ms)  # registers1/2 cannot hold L = 1024
    assert "registers1" not in ms
    assert tune.tune(1024, 5, precision="fp32", cache_file=f)[0] == best  # cached


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp32", "fx64"])
def test_tuner_times_the_cluster_sweeps_on_long_chains(plr, precision):
    """At L = 8192 no single CTA's registers hold a slot: the tuner times the
    global-memory sweep and both cluster sweeps (shared memory and registers of
    a cluster of CTAs) and picks the fastest of those it timed."""
    from paper_1308_5426_gb300 import tune
    best, ms = tune.tune(8192, 5, sigma=0.5, precision=precision, R=8, sweeps=2, warm=1)
    assert {"global", "cluster", "rcluster"} <= set(ms)
    assert not any(v.startswith("registers") for v in ms)
    assert best in ms and ms[best] == min(ms.values())
