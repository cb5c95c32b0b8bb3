"""Batching: ragged jobs (different L, q, sigma, R, precision) stepped together
in graph-captured batch steps give each job exactly the results it gets alone
with the same call sequence (bit for bit), and FP64 jobs in a batch still
follow the oracle."""
import numpy as np
import pytest

import oracle
from paper_1308_5426_gb300 import workloads

pytestmark = pytest.mark.gpu

JOBS = [  # L, q, sigma, R, seed, precision, K
    (64, 3, 0.5, 16, 1, "fp64", 0),
    (100, 7, 0.3, 5, 2, "fp32", 10),
    (1000, 5, 0.4, 6, 3, "fp64", 0),
    (300, 4, 0.8, 9, 4, "fp32", 7),
    (4096, 8, 0.2, 3, 5, "fp32", 6),
    (33, 16, 0.9, 1, 6, "fp64", 0),
]


@pytest.fixture(scope="module")
def plr():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1308_5426_gb300
    return paper_1308_5426_gb300


def _make(plr, spec, stream=None):
    L, q, sigma, R, seed, prec, K = spec
    temps = workloads.geometric_ratios(R, 0.05, 1.0) * oracle.jtot(L, sigma)
    return plr.Job(L, q, sigma, temps, seed, precision=prec, recompute_every=K, stream=stream)


@pytest.mark.parametrize("steps,per_graph", [(23, 10), (7, 3)])
def test_batch_equals_alone(plr, steps, per_graph):
    alone = []
    for spec in JOBS:
        j = _make(plr, spec)
        for _ in range(steps):
            j.sweep(1)
            j.exchange()
        alone.append((j.spins(), j.running_energy(), j.fields(), j.measure(), j.stats()))
        j.close()
    jobs = [_make(plr, spec) for spec in JOBS]
    b = plr.Batch(jobs)
    b.run(steps, per_graph)
    b.sync()
    Eb, Mb = b.measure()
    off = 0
    for spec, j, (S, E, F, (Em, Mm), st) in zip(JOBS, jobs, alone):
        np.testing.assert_array_equal(j.spins(), S, err_msg=str(spec))
        np.testing.assert_array_equal(j.running_energy(), E, err_msg=str(spec))
        np.testing.assert_array_equal(j.fields(), F, err_msg=str(spec))
        np.testing.assert_array_equal(Eb[off:off + j.R], Em, err_msg=str(spec))
        np.testing.assert_array_equal(Mb[off:off + j.R], Mm, err_msg=str(spec))
        np.testing.assert_array_equal(j.stats()["acc_flip"], st["acc_flip"])
        assert j.counters() == (steps, steps)
        off += j.R
    b.close()


def test_batch_fp64_jobs_follow_oracle(plr):
    specs = [s for s in JOBS if s[5] == "fp64"]
    jobs = [_make(plr, s) for s in specs]
    b = plr.Batch(jobs)
    b.run(12, 5)
    b.sync()
    for s, j in zip(specs, jobs):
        L, q, sigma, R, seed, _, _ = s
        temps = workloads.geometric_ratios(R, 0.05, 1.0) * oracle.jtot(L, sigma)
        o = oracle.Oracle(L, q, sigma, temps, seed)
        for _ in range(12):
            o.step()
        assert o.stats()["near_metro"].sum() == 0
        np.testing.assert_array_equal(j.spins(), o.spins(), err_msg=str(s))


def test_batch_split_calls_equal_run(plr):
    """batch.sweep + batch.exchange alternated equal batch.run."""
    a = [_make(plr, s) for s in JOBS[:4]]
    b = [_make(plr, s) for s in JOBS[:4]]
    ba, bb = plr.Batch(a), plr.Batch(b)
    ba.run(9, 4)
    for _ in range(9):
        bb.sweep(1)
        bb.exchange()
    ba.sync()
    bb.sync()
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x.spins(), y.spins())
        np.testing.assert_array_equal(x.fields(), y.fields())


def test_batch_checkpoint_resume(plr):
    """potts_lr_batch_get_state / set_state: the batch checkpoint is the jobs'
    own checkpoints back to back; restoring it and re-running the same steps
    reproduces every job bit for bit; a corrupt part is refused before any job
    changes (a long FP32 job on the cluster kernel included)."""
    specs = JOBS + [(10000, 7, 0.5, 2, 7, "fp32", 4)]
    jobs = [_make(plr, s) for s in specs]
    b = plr.Batch(jobs)
    b.run(5, 5)
    b.sync()
    state = b.get_state()
    assert len(state) == b.state_size()
    assert state == b"".join(j.get_state() for j in jobs)

    def snapshot():
        return [(j.spins(), j.fields(), j.running_energy(), j.stats()["acc_flip"]) for j in jobs]

    b.run(6, 3)
    b.sync()
    first = snapshot()
    b.set_state(state)
    b.run(6, 3)
    b.sync()
    again = snapshot()
    for x, y in zip(first, again):
        for u, v in zip(x, y):
            np.testing.assert_array_equal(u, v)

    # a corrupt slot map in the last job's part (the map follows the 72-byte
    # header: magic, version, L, q, R, precision, c, Lpad, seed, nsweep,
    # nexch, sigma bits, temperature hash, FX64 grid, reserved): refused,
    # nothing changes
    bad = bytearray(state)
    off = len(state) - len(jobs[-1].get_state())  # the last part starts here
    before = snapshot()
    import struct
    from paper_1308_5426_gb300 import _lib
    bad[off + 72:off + 80] = struct.pack("<ii", 0, 0)  # slots 0 and 1 -> replica 0 twice
    with pytest.raises(plr.PottsError) as e:
        b.set_state(bytes(bad))
    assert e.value.code == _lib.ESTATE
    bad = bytearray(state)
    bad[off + 4:off + 8] = struct.pack("<I", 3)  # an older format version
    with pytest.raises(plr.PottsError):
        b.set_state(bytes(bad))
    after = snapshot()
    for x, y in zip(before, after):
        for u, v in zip(x, y):
            np.testing.assert_array_equal(u, v)
    b.close()
    for j in jobs:
        j.close()


def test_crowded_batch_equals_alone(plr):
    """40 jobs of L = 6000, q = 4, R = 64 (2560 slots, more than 16 per SM):
    alone each sweeps on a CTA cluster (94 KB of fields per slot), in the
    crowded batch on one CTA per slot; spins, fields and energies agree bit for
    bit."""
    L, q, sigma, R, n = 6000, 4, 0.5, 64, 40
    temps = workloads.geometric_ratios(R, 0.05, 1.0) * oracle.jtot(L, sigma)
    alone = [plr.Job(L, q, sigma, temps, 100 + i, precision="fp32", recompute_every=0) for i in range(n)]
    for j in alone:
        for _ in range(3):
            j.sweep(1)
            j.exchange()
    batched = [plr.Job(L, q, sigma, temps, 100 + i, precision="fp32", recompute_every=0) for i in range(n)]
    b = plr.Batch(batched)
    b.run(3, 3)
    b.sync()
    for x, y in zip(alone, batched):
        np.testing.assert_array_equal(x.spins(), y.spins())
        np.testing.assert_array_equal(x.fields(), y.fields())
        np.testing.assert_array_equal(x.running_energy(), y.running_energy())
    b.close()
    for j in alone + batched:
        j.close()


def test_crowded_batch_takes_the_smallest_automatic_cluster(plr):
    """An FP64 job whose automatic cluster is larger than its fields need
    (L = 4096, q = 8, R = 3: 8 CTAs alone, 2 needed) sweeps on the smallest
    cluster inside a batch of more than 16 slots per SM (filled with small FP32
    jobs); its spins, fields and energies equal the job run alone."""
    import torch
    nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    L, q, sigma, R = 4096, 8, 0.2, 3
    temps = workloads.geometric_ratios(R, 0.05, 1.0) * oracle.jtot(L, sigma)
    alone = plr.Job(L, q, sigma, temps, 41, precision="fp64")
    assert alone.sweep_info()["cluster"] > plr.Job(L, q, sigma, temps, 41, precision="fp64",
                                                   sweep_variant="cluster").sweep_info()["cluster"]
    for _ in range(3):
        alone.sweep(1)
        alone.exchange()
    nsmall = (16 * nsm) // 64 + 1
    small_temps = workloads.geometric_ratios(64, 0.05, 1.0) * oracle.jtot(64, 0.5)
    small = [plr.Job(64, 2, 0.5, small_temps, 300 + i, precision="fp32", recompute_every=0) for i in range(nsmall)]
    big = plr.Job(L, q, sigma, temps, 41, precision="fp64")
    b = plr.Batch([big] + small)
    b.run(3, 3)
    b.sync()
    np.testing.assert_array_equal(alone.spins(), big.spins())
    np.testing.assert_array_equal(alone.fields(), big.fields())
    np.testing.assert_array_equal(alone.running_energy(), big.running_energy())
    b.close()
    for j in [alone, big] + small:
        j.close()


def test_batch_of_many_slots_gives_8byte_jobs_one_cta_per_slot(plr):
    """FP64 jobs of L = 4096, q = 5, R = 64 (160 KB of fields, which fit one
    CTA) take a cluster alone; ten of them in one batch (640 slots, more than
    four per SM) sweep one CTA per slot, the fields in its shared memory.
    Spins, fields and energies equal each job run alone."""
    import torch
    nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    L, q, sigma, R = 4096, 5, 0.85, 64
    n = (4 * nsm) // R + 1
    temps = workloads.geometric_ratios(R, 0.05, 1.0) * oracle.jtot(L, sigma)
    alone = [plr.Job(L, q, sigma, temps, 500 + i, precision="fp64") for i in range(n)]
    assert all(j.sweep_info()["kernel"] == "cluster" for j in alone)
    for j in alone:
        for _ in range(2):
            j.sweep(1)
            j.exchange()
    batched = [plr.Job(L, q, sigma, temps, 500 + i, precision="fp64") for i in range(n)]
    b = plr.Batch(batched)
    b.run(2, 2)
    b.sync()
    for x, y in zip(alone, batched):
        np.testing.assert_array_equal(x.spins(), y.spins())
        np.testing.assert_array_equal(x.fields(), y.fields())
        np.testing.assert_array_equal(x.running_energy(), y.running_energy())
    b.close()
    for j in alone + batched:
        j.close()


def test_random_site_job_keeps_the_direct_sweep_in_a_batch_of_many_slots(plr):
    """An FP64 job with random site order (the direct sweep) whose fields would
    take a cluster (L = 2048, q = 5: 80 KB) keeps the direct sweep inside a
    batch of more than four slots per SM; its spins and energies equal the job
    run alone."""
    import torch
    nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    L, q, sigma, R = 2048, 5, 0.5, 64
    temps = workloads.geometric_ratios(R, 0.05, 1.0) * oracle.jtot(L, sigma)
    alone = plr.Job(L, q, sigma, temps, 61, precision="fp64", site_order="random")
    assert alone.sweep_info()["kernel"] == "direct"
    for _ in range(2):
        alone.sweep(1)
        alone.exchange()
    nsmall = (4 * nsm) // 64 + 1
    small_temps = workloads.geometric_ratios(64, 0.05, 1.0) * oracle.jtot(64, 0.5)
    small = [plr.Job(64, 2, 0.5, small_temps, 700 + i, precision="fp64") for i in range(nsmall)]
    job = plr.Job(L, q, sigma, temps, 61, precision="fp64", site_order="random")
    b = plr.Batch([job] + small)
    b.run(2, 2)
    b.sync()
    np.testing.assert_array_equal(alone.spins(), job.spins())
    np.testing.assert_array_equal(alone.running_energy(), job.running_energy())
    b.close()
    for j in [alone, job] + small:
        j.close()
