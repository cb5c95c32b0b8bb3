"""Failure handling on the GPU, without faulting it: checkpoints that do not
belong to a job are refused before any device memory changes; bounded device
waits that are made to expire (by setting their limits to zero) end in an
error status the host reads, with the context still usable; and the SM
placement wait, whose expiry only changes which SM sweeps which slot,
changes no result when it expires."""
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


def _job(plr, L=96, q=4, sigma=0.5, R=6, seed=11, c=2, precision="fp64", ratios=None):
    ratios = workloads.geometric_ratios(R, 0.05, 1.0) if ratios is None else ratios
    temps = np.asarray(ratios) * oracle.jtot(L, sigma)
    return plr.Job(L, q, sigma, temps, seed, precision=precision, pair_factor=c)


@pytest.mark.parametrize("precision", ["fp64", "fx64", "fp32"])
def test_checkpoint_of_another_job_is_refused(plr, precision):
    """A checkpoint restores only into a job with the same L, q, sigma,
    temperatures, R, seed, precision and pair factor: anything else would
    continue with fields of other couplings, another chain or another energy
    scale, so it is refused with ESTATE and the job is left as it was."""
    from paper_1308_5426_gb300 import _lib
    a = _job(plr, precision=precision)
    for _ in range(5):
        a.sweep(1)
        a.exchange()
    st = a.get_state()
    others = {
        "sigma": _job(plr, sigma=0.55, precision=precision),
        "seed": _job(plr, seed=12, precision=precision),
        "pair factor": _job(plr, c=1, precision=precision),
        "temperatures": _job(plr, ratios=workloads.geometric_ratios(6, 0.05, 0.9), precision=precision),
    }
    for what, b in others.items():
        before = (b.spins(), b.fields(), b.running_energy())
        with pytest.raises(plr.PottsError) as e:
            b.set_state(st)
        assert e.value.code == _lib.ESTATE, what
        after = (b.spins(), b.fields(), b.running_energy())
        for x, y in zip(before, after):
            np.testing.assert_array_equal(x, y, err_msg=what)
        b.close()
    same = _job(plr, precision=precision)
    same.set_state(st)
    np.testing.assert_array_equal(same.spins(), a.spins())
    same.close()
    a.close()


def test_rebuild_wait_expiry_reports_timeout_and_recovers(plr):
    """With the rebuild's wait bound at zero, the first pipeline wait that is
    not already complete expires: the rebuild stops, drains its own copies and
    tensor-core work, frees its tensor memory and returns, and the next
    synchronising call reports ETIMEOUT.  With the bound restored, a rebuild
    gives fields equal to the oracle's again, and the job runs on."""
    from paper_1308_5426_gb300 import _lib
    L, q, sigma, R, seed = 1024, 5, 0.4, 16, 3
    ratios = workloads.geometric_ratios(R, 0.05, 1.0)
    temps = ratios * oracle.jtot(L, sigma)
    g = plr.Job(L, q, sigma, temps, seed, precision="fp32", recompute_every=0)
    g.sweep(3)
    g.sync()
    g.set_wait_limits(rebuild_ns=0)
    g.fields_recompute()
    with pytest.raises(plr.PottsError) as e:
        g.sync()
    assert e.value.code == _lib.ETIMEOUT
    g.sync()  # the status was read and cleared; the context is still usable
    g.set_wait_limits()  # defaults
    g.fields_recompute()
    g.sync()
    o = oracle.Oracle(L, q, sigma, temps, seed)
    o.set_spins(g.spins())
    jt = oracle.jtot(L, sigma)
    np.testing.assert_allclose(g.fields(), o.fields(), rtol=0, atol=1e-6 * jt)
    assert g.fields_error() < 1e-6
    g.sweep(2)
    g.exchange()
    g.sync()
    g.close()


def test_plan_wait_expiry_changes_no_result(plr):
    """More slots than SMs engage the placement plan; with its wait bound at
    zero the CTAs take items without waiting for the others' first claims.
    The results are those of the default run, and the oracle's."""
    L, q, sigma, R, seed = 64, 3, 0.5, 400, 2
    ratios = workloads.geometric_ratios(R, 0.05, 1.0)
    temps = ratios * oracle.jtot(L, sigma)
    a = plr.Job(L, q, sigma, temps, seed)
    b = plr.Job(L, q, sigma, temps, seed)
    b.set_wait_limits(plan_ns=0)
    o = oracle.Oracle(L, q, sigma, temps, seed)
    for _ in range(8):
        a.sweep(1)
        a.exchange()
        b.sweep(1)
        b.exchange()
        o.step()
    np.testing.assert_array_equal(a.spins(), b.spins())
    np.testing.assert_array_equal(a.running_energy(), b.running_energy())
    np.testing.assert_array_equal(b.spins(), o.spins())
    a.close()
    b.close()
