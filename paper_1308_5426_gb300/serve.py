"""Continuous-batching service for parallel-tempering jobs on one GPU.

Requests (phase-diagram points: q, sigma, L, temperature grid, seed, sweeps)
arrive over time.  The loop admits queued requests, first come first served,
while their field memory (L q R w bytes: w = 4 for the FP32 local fields of
the served mixed-precision jobs, 8 for FP64 or FX64 fields) fits in the
budget; every active job keeps its spins and fields on the device between
chunks; each chunk runs `chunk` batch steps (one sweep of every slot of every
active job + one exchange step per job) as one graph-captured batch, then
measures every active job.  Jobs leave when their sweeps are done, freeing
memory for the queue.  Because every job's random numbers are keyed by its own
seed, slot, sweep and site, and a job's kernels never depend on its neighbours
in the batch, each job's results are identical alone and in the mix.

The GPU work goes through the library's C ABI (Job, Batch); the scheduling is
plain host code behind a small engine interface so that it can be exercised
without a GPU.
"""
import time
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional

import numpy as np


@dataclass
class Request:
    rid: int
    L: int
    q: int
    sigma: float
    temps: np.ndarray
    seed: int
    sweeps: int
    precision: str = "fp32"
    recompute_every: int = 100
    arrival: float = 0.0

    @property
    def R(self) -> int:
        return int(len(self.temps))

    @property
    def footprint(self) -> int:
        """Admission footprint: the field memory L q R w bytes, w the field
        word (4 bytes in FP32 mode, 8 in FP64 and FX64 modes)."""
        return self.L * self.q * self.R * (4 if self.precision == "fp32" else 8)

    @property
    def attempts(self) -> int:
        return self.L * self.R * self.sweeps


@dataclass
class Result:
    rid: int
    status: str                     # "done", "rejected", "cancelled", "failed"
    arrival: float = 0.0
    admitted: Optional[float] = None
    finished: Optional[float] = None
    sweeps_done: int = 0
    at: List[int] = field(default_factory=list)        # sweeps done at each measurement
    E: List[np.ndarray] = field(default_factory=list)  # per measurement: energies per slot
    M: List[np.ndarray] = field(default_factory=list)
    spins: Optional[np.ndarray] = None                 # final spins (keep_spins)
    error: str = ""

    @property
    def latency(self) -> Optional[float]:
        return None if self.finished is None else self.finished - self.arrival

    def observables(self, L: int, nblocks: int = 20, skip: int = 0):
        """<E>/L, <M>, U_E (Eq. 11) and V_M (Eq. 12) per slot with jackknife
        errors, from the measurements after the first `skip` ones."""
        from .analysis import observables
        return observables(np.array(self.E[skip:]), np.array(self.M[skip:]), L, nblocks)


class GpuEngine:
    """The library's C ABI as the service's engine."""

    def __init__(self, stream=None, variants=None):
        """variants: optional {(L, q, precision): sweep variant name}, e.g.
        from tune.tune() run over the shapes a trace will bring."""
        import paper_1308_5426_gb300 as plr
        self.plr = plr
        self.stream = stream
        self.variants = dict(variants or {})

    def create(self, req: Request):
        v = self.variants.get((req.L, req.q, req.precision), "auto")
        return self.plr.Job(req.L, req.q, req.sigma, req.temps, req.seed, precision=req.precision,
                            recompute_every=req.recompute_every, stream=self.stream, sweep_variant=v)

    def batch(self, jobs):
        return self.plr.Batch(jobs, stream=self.stream)

    def run(self, batch, nsteps: int):
        batch.run(nsteps, nsteps)

    def measure(self, batch):
        return batch.measure()

    def destroy_batch(self, batch):
        batch.close()

    def spins(self, job):
        return job.spins()

    def destroy(self, job):
        job.close()


class Server:
    """Admit, batch, step and retire jobs; `clock` gives seconds since start."""

    def __init__(self, engine, budget_bytes: int, chunk: int = 10, clock: Callable[[], float] = None,
                 keep_spins: bool = False):
        if chunk < 1:
            raise ValueError("chunk must be >= 1")
        self.keep_spins = keep_spins
        self.engine = engine
        self.budget = int(budget_bytes)
        self.chunk = int(chunk)
        t0 = time.perf_counter()
        self.clock = clock or (lambda: time.perf_counter() - t0)
        self.queue: List[Request] = []
        self.active: Dict[int, tuple] = {}   # rid -> (request, job)
        self.results: Dict[int, Result] = {}
        self.used = 0
        self._batch = None
        self._batch_ids = ()
        self.attempts_done = 0
        self.busy_seconds = 0.0

    # ---- requests
    def submit(self, req: Request):
        if req.rid in self.results or any(r.rid == req.rid for r in self.queue) or req.rid in self.active:
            raise ValueError("duplicate request id %d" % req.rid)
        res = Result(rid=req.rid, status="queued", arrival=req.arrival)
        self.results[req.rid] = res
        if req.footprint > self.budget:
            res.status = "rejected"
            res.error = "footprint %d B exceeds the budget %d B" % (req.footprint, self.budget)
            return res
        self.queue.append(req)
        return res

    def cancel(self, rid: int):
        """Drop a queued or running job between chunks; the others are unaffected."""
        for i, r in enumerate(self.queue):
            if r.rid == rid:
                del self.queue[i]
                self.results[rid].status = "cancelled"
                return True
        if rid in self.active:
            req, job = self.active.pop(rid)
            self._drop_batch()
            self.engine.destroy(job)
            self.used -= req.footprint
            self.results[rid].status = "cancelled"
            return True
        return False

    # ---- loop
    def _drop_batch(self):
        if self._batch is not None:
            self.engine.destroy_batch(self._batch)
            self._batch = None
            self._batch_ids = ()

    def _admit(self, now: float):
        admitted = False
        while self.queue and self.queue[0].arrival <= now and self.used + self.queue[0].footprint <= self.budget:
            req = self.queue.pop(0)
            res = self.results[req.rid]
            try:
                job = self.engine.create(req)
            except Exception as e:  # a failed create leaves every other job untouched
                res.status = "failed"
                res.error = str(e)
                continue
            self.active[req.rid] = (req, job)
            self.used += req.footprint
            res.status = "running"
            res.admitted = now
            admitted = True
        return admitted

    def step(self) -> bool:
        """Admit what fits, run one chunk of the active jobs, retire finished
        ones.  Returns False when nothing is active or queued."""
        now = self.clock()
        if self._admit(now):
            self._drop_batch()
        if not self.active:
            return bool(self.queue)
        ids = tuple(sorted(self.active))
        n = min(self.chunk, min(self.active[i][0].sweeps - self.results[i].sweeps_done for i in ids))
        t0 = time.perf_counter()
        try:
            if self._batch is None or self._batch_ids != ids:
                self._drop_batch()
                self._batch = self.engine.batch([self.active[i][1] for i in ids])
                self._batch_ids = ids
            self.engine.run(self._batch, n)
            E, M = self.engine.measure(self._batch)
        except Exception as e:
            # an engine failure (batch set-up, step or measurement) fails the
            # jobs of this chunk, not the service
            if self._batch is not None:
                try:
                    self.engine.destroy_batch(self._batch)
                except Exception:
                    pass
            for i in ids:
                req, job = self.active.pop(i)
                self.results[i].status = "failed"
                self.results[i].error = str(e)
                self.used -= req.footprint
                try:
                    self.engine.destroy(job)
                except Exception:
                    pass
            self._batch = None
            self._batch_ids = ()
            return True
        self.busy_seconds += time.perf_counter() - t0
        off = 0
        done = []
        for i in ids:
            req, _ = self.active[i]
            res = self.results[i]
            res.sweeps_done += n
            res.at.append(res.sweeps_done)
            res.E.append(np.array(E[off:off + req.R]))
            res.M.append(np.array(M[off:off + req.R]))
            off += req.R
            self.attempts_done += req.L * req.R * n
            if res.sweeps_done >= req.sweeps:
                done.append(i)
        if done:
            t = self.clock()
            self._drop_batch()
            for i in done:
                req, job = self.active.pop(i)
                if self.keep_spins:
                    self.results[i].spins = self.engine.spins(job)
                self.engine.destroy(job)
                self.used -= req.footprint
                self.results[i].status = "done"
                self.results[i].finished = t
        return True

    def run(self, requests: List[Request], idle_sleep: float = 1e-3, timeout: float = None):
        """Serve a trace: requests are submitted when the clock reaches their
        arrival time; returns when every request has a final status."""
        pending = sorted(requests, key=lambda r: r.arrival)
        t_start = self.clock()
        while True:
            now = self.clock()
            while pending and pending[0].arrival <= now:
                self.submit(pending.pop(0))
            busy = self.step()
            if not pending and not self.queue and not self.active:
                break
            if not busy:
                if pending:
                    time.sleep(max(0.0, min(idle_sleep, pending[0].arrival - self.clock())))
            if timeout is not None and self.clock() - t_start > timeout:
                raise TimeoutError("service did not drain within %.1f s" % timeout)
        self._drop_batch()
        return self.results

    def summary(self, wall_seconds: float = None):
        lat = np.array([r.latency for r in self.results.values() if r.status == "done"])
        out = {"done": int(lat.size),
               "rejected": sum(r.status == "rejected" for r in self.results.values()),
               "failed": sum(r.status == "failed" for r in self.results.values()),
               "cancelled": sum(r.status == "cancelled" for r in self.results.values()),
               "attempts": int(self.attempts_done)}
        if lat.size:
            out["p50_s"] = float(np.percentile(lat, 50))
            out["p99_s"] = float(np.percentile(lat, 99))
        if wall_seconds:
            out["attempts_per_s"] = self.attempts_done / wall_seconds
        if self.busy_seconds > 0:
            out["attempts_per_busy_s"] = self.attempts_done / self.busy_seconds
        return out
