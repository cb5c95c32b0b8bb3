"""Continuous batching on the GPU: jobs arriving while others run are admitted
as memory frees up, share batch steps with them, and still produce exactly the
results they produce alone (every measurement at the same sweep count, and the
final spins, bit for bit)."""
import numpy as np
import pytest

import oracle
from paper_1308_5426_gb300 import workloads
from paper_1308_5426_gb300.serve import GpuEngine, Request, Server

pytestmark = pytest.mark.gpu

SPECS = [  # L, q, sigma, R, sweeps, arrival
    (256, 3, 0.5, 8, 60, 0.00),
    (1024, 5, 0.4, 6, 40, 0.00),
    (512, 8, 0.8, 4, 70, 0.02),
    (64, 3, 0.2, 16, 30, 0.03),
    (2048, 4, 0.6, 5, 50, 0.05),
    (300, 6, 0.3, 7, 45, 0.06),
]


class StepClock:
    """Deterministic clock: 0.01 s per call."""

    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 0.01
        return self.t


def _requests():
    out = []
    for i, (L, q, sigma, R, sweeps, arr) in enumerate(SPECS):
        temps = workloads.geometric_ratios(R, 0.05, 1.0) * oracle.jtot(L, sigma)
        out.append(Request(rid=i, L=L, q=q, sigma=sigma, temps=temps, seed=100 + i, sweeps=sweeps,
                           recompute_every=20, arrival=arr))
    return out


LONG_SPECS = [  # L, q, sigma, R, sweeps, arrival, precision: requests that take the cluster kernels
    (16384, 5, 0.4, 4, 12, 0.00, "fp32"),   # FP32 fields in the registers of a 4-CTA cluster
    (8192, 3, 0.6, 5, 15, 0.00, "fp32"),    # one CTA's registers (26 sites per thread)
    (10000, 16, 0.5, 3, 10, 0.02, "fp32"),  # q > 12: the shared memory of a cluster
    (9000, 5, 0.3, 3, 10, 0.03, "fx64"),    # FX64 fields in the registers of a 4-CTA cluster
    (6000, 5, 0.7, 3, 8, 0.04, "fp64"),     # FP64 fields in the shared memory of a cluster (2 CTAs needed)
]


def _long_requests():
    out = []
    for i, (L, q, sigma, R, sweeps, arr, prec) in enumerate(LONG_SPECS):
        temps = workloads.geometric_ratios(R, 0.05, 1.0) * oracle.jtot(L, sigma)
        out.append(Request(rid=i, L=L, q=q, sigma=sigma, temps=temps, seed=200 + i, sweeps=sweeps,
                           precision=prec, recompute_every=4, arrival=arr))
    return out


@pytest.mark.parametrize("which", ["short", "long"])
def test_served_results_equal_alone(which):
    import __graft_entry__
    __graft_entry__.build()
    import paper_1308_5426_gb300 as plr
    reqs = _requests() if which == "short" else _long_requests()
    budget = int(2.2 * max(r.footprint for r in reqs))  # forces queueing
    srv = Server(GpuEngine(), budget_bytes=budget, chunk=10 if which == "short" else 4, clock=StepClock(),
                 keep_spins=True)
    res = srv.run(reqs, idle_sleep=0.0)
    assert all(r.status == "done" for r in res.values())
    # at least one job was admitted after another had started running
    starts = sorted(r.admitted for r in res.values())
    assert starts[-1] > starts[0]
    for r in reqs:
        out = res[r.rid]
        job = plr.Job(r.L, r.q, r.sigma, r.temps, r.seed, precision=r.precision,
                      recompute_every=r.recompute_every)
        if which == "long":
            want = {0: "register_cluster", 1: "registers", 2: "cluster", 3: "register_cluster", 4: "cluster"}
            assert job.sweep_info()["kernel"] == want[r.rid], (r.rid, job.sweep_info())
        done = 0
        for at, E, M in zip(out.at, out.E, out.M):
            while done < at:
                job.sweep(1)
                job.exchange()
                done += 1
            Ea, Ma = job.measure()
            np.testing.assert_array_equal(E, Ea, err_msg="job %d at sweep %d" % (r.rid, at))
            np.testing.assert_array_equal(M, Ma, err_msg="job %d at sweep %d" % (r.rid, at))
        assert done == r.sweeps
        np.testing.assert_array_equal(out.spins, job.spins())
        job.close()
    s = srv.summary()
    assert s["done"] == len(reqs) and s["p99_s"] >= s["p50_s"] > 0
