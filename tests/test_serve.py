"""Host logic of the continuous-batching service (no GPU): admission by field
footprint, first-come-first-served order, the memory budget, chunking,
cancellation, rejected and failing requests -- each failure leaves the other
jobs' results unchanged.  The engine is a deterministic fake whose
'measurement' of a job is a function of its seed and sweep count only."""
import numpy as np
import pytest

from paper_1308_5426_gb300.serve import Request, Server


class FakeJob:
    def __init__(self, req):
        self.req = req
        self.sweeps = 0


class FakeEngine:
    def __init__(self, fail_seeds=(), fail_run_at=None, fail_batch_at=None):
        self.fail_seeds = set(fail_seeds)
        self.fail_run_at = fail_run_at
        self.fail_batch_at = fail_batch_at
        self.runs = 0
        self.live = set()
        self.max_live_bytes = 0
        self.batches = 0
        self.batches_destroyed = 0

    def create(self, req):
        if req.seed in self.fail_seeds:
            raise RuntimeError("create failed for seed %d" % req.seed)
        j = FakeJob(req)
        self.live.add(j)
        self.max_live_bytes = max(self.max_live_bytes, sum(x.req.footprint for x in self.live))
        return j

    def batch(self, jobs):
        if self.fail_batch_at is not None and self.batches + 1 == self.fail_batch_at:
            self.fail_batch_at = None
            raise RuntimeError("batch set-up failed")
        self.batches += 1
        return list(jobs)

    def run(self, batch, n):
        self.runs += 1
        if self.fail_run_at is not None and self.runs == self.fail_run_at:
            raise RuntimeError("device step failed")
        for j in batch:
            j.sweeps += n

    def measure(self, batch):
        E = np.concatenate([np.full(j.req.R, 1000.0 * j.req.seed + j.sweeps) for j in batch])
        return E, -E

    def destroy_batch(self, batch):
        self.batches_destroyed += 1

    def destroy(self, job):
        self.live.discard(job)

    def spins(self, job):
        return np.full((job.req.R, job.req.L), job.sweeps % 7, np.uint8)


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 0.01
        return self.t


def _req(rid, L=64, q=3, R=4, sweeps=30, arrival=0.0, seed=None):
    return Request(rid=rid, L=L, q=q, sigma=0.5, temps=np.linspace(1, 2, R), seed=rid + 1 if seed is None else seed,
                   sweeps=sweeps, arrival=arrival)


def test_all_jobs_complete_with_their_own_results():
    eng = FakeEngine()
    srv = Server(eng, budget_bytes=10 ** 9, chunk=10, clock=Clock())
    reqs = [_req(i, sweeps=10 * (i + 1), arrival=0.05 * i) for i in range(5)]
    res = srv.run(reqs, idle_sleep=0.0)
    for r in reqs:
        out = res[r.rid]
        assert out.status == "done" and out.sweeps_done == r.sweeps
        assert out.at[-1] == r.sweeps
        np.testing.assert_array_equal(out.E[-1], 1000.0 * r.seed + r.sweeps)
        assert out.latency > 0
    s = srv.summary(wall_seconds=1.0)
    assert s["done"] == 5 and s["attempts"] == sum(r.attempts for r in reqs)
    assert "p50_s" in s and "p99_s" in s and s["p99_s"] >= s["p50_s"]


def test_admission_respects_budget_and_order():
    eng = FakeEngine()
    one = _req(0).footprint
    srv = Server(eng, budget_bytes=2 * one, chunk=10, clock=Clock())
    reqs = [_req(i, sweeps=20) for i in range(6)]
    res = srv.run(reqs, idle_sleep=0.0)
    assert eng.max_live_bytes <= 2 * one
    adm = [res[i].admitted for i in range(6)]
    assert adm == sorted(adm)  # first come, first served
    assert all(res[i].status == "done" for i in range(6))


def test_oversized_request_rejected_others_served():
    eng = FakeEngine()
    small = _req(0)
    srv = Server(eng, budget_bytes=small.footprint * 3, chunk=10, clock=Clock())
    reqs = [small, _req(1, L=4096, q=16, R=64), _req(2)]
    res = srv.run(reqs, idle_sleep=0.0)
    assert res[1].status == "rejected" and "budget" in res[1].error
    for i in (0, 2):
        assert res[i].status == "done"
        np.testing.assert_array_equal(res[i].E[-1], 1000.0 * reqs[i].seed + reqs[i].sweeps)


def test_failing_create_leaves_others_unchanged():
    eng = FakeEngine(fail_seeds={99})
    srv = Server(eng, budget_bytes=10 ** 9, chunk=10, clock=Clock())
    reqs = [_req(0), _req(1, seed=99), _req(2)]
    res = srv.run(reqs, idle_sleep=0.0)
    assert res[1].status == "failed" and "create failed" in res[1].error
    assert res[0].status == "done" and res[2].status == "done"


def test_cancel_running_job_between_chunks():
    eng = FakeEngine()
    srv = Server(eng, budget_bytes=10 ** 9, chunk=10, clock=Clock())
    for i in range(3):
        srv.submit(_req(i, sweeps=50))
    srv.step()
    srv.step()
    assert srv.cancel(1)
    assert not srv.cancel(1)
    while srv.step():
        pass
    res = srv.results
    assert res[1].status == "cancelled" and res[1].sweeps_done == 20
    for i in (0, 2):
        assert res[i].status == "done" and res[i].sweeps_done == 50
        np.testing.assert_array_equal(res[i].E[-1], 1000.0 * (i + 1) + 50)
    assert len(eng.live) == 0 and srv.used == 0


def test_engine_failure_fails_that_chunk_only():
    eng = FakeEngine(fail_run_at=2)
    srv = Server(eng, budget_bytes=_req(0).footprint, chunk=10, clock=Clock())
    reqs = [_req(0, sweeps=30), _req(1, sweeps=30)]
    res = srv.run(reqs, idle_sleep=0.0)
    assert res[0].status == "failed" and "device step failed" in res[0].error
    assert res[1].status == "done" and res[1].sweeps_done == 30
    assert srv.used == 0


def test_duplicate_ids_refused():
    srv = Server(FakeEngine(), budget_bytes=10 ** 9)
    srv.submit(_req(0))
    with pytest.raises(ValueError):
        srv.submit(_req(0))


def test_footprint_follows_the_field_word():
    """Admission counts 4-byte FP32 fields and 8-byte FP64 / FX64 fields."""
    r32 = _req(0, L=100, q=5, R=8)
    assert r32.footprint == 100 * 5 * 8 * 4
    for prec in ("fp64", "fx64"):
        r = Request(rid=1, L=100, q=5, sigma=0.5, temps=np.ones(8), seed=1, sweeps=1, precision=prec)
        assert r.footprint == 100 * 5 * 8 * 8
    # a budget that holds the FP32 form of a request but not its FP64 form
    srv = Server(FakeEngine(), budget_bytes=100 * 5 * 8 * 4, chunk=5, clock=Clock())
    assert srv.submit(Request(rid=2, L=100, q=5, sigma=0.5, temps=np.ones(8), seed=1, sweeps=1,
                              precision="fp64")).status == "rejected"
    assert srv.submit(_req(3, L=100, q=5, R=8)).status == "queued"


def test_failed_step_releases_its_batch():
    """A failing device step destroys the chunk's batch as well as its jobs."""
    eng = FakeEngine(fail_run_at=2)
    srv = Server(eng, budget_bytes=10 ** 9, chunk=10, clock=Clock())
    srv.run([_req(0, sweeps=50), _req(1, sweeps=50)], idle_sleep=0.0)
    assert eng.batches == eng.batches_destroyed
    assert not eng.live and srv.used == 0


def test_failed_batch_setup_fails_only_that_chunk():
    """A batch that cannot be set up fails the jobs it would have held; jobs
    that arrive later are served normally."""
    eng = FakeEngine(fail_batch_at=1)
    srv = Server(eng, budget_bytes=10 ** 9, chunk=10, clock=Clock())
    res = srv.run([_req(0, sweeps=20), _req(1, sweeps=20, arrival=0.5)], idle_sleep=0.0)
    assert res[0].status == "failed" and "batch set-up" in res[0].error
    assert res[1].status == "done" and res[1].sweeps_done == 20
    assert not eng.live and srv.used == 0
