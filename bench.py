"""Benchmark: spin-flip attempts/s of parallel-tempering Metropolis on the
long-range q-state Potts chain (arXiv:1308.5426), one JSON line on rank 0.

Default workload: eight independent plain-FP64 PT chains, L=1024, q=5,
sigma=0.4, R=64 temperatures geometric in T/Jtot in [0.05, 1], seeds 1..8,
energy and magnetisation measured every 10 sweeps.  One step = 10 x (one sweep
of every slot + one exchange step) + one measurement, over all 8 chains.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload chains|precision|batching|serving|paper]

Beside the main line (the eight chains in FP64), the default run adds one key
per workload of the method's contract, each timed with CUDA events on its own
stream: the precision job (L=4096 q=8 R=128) in FP32, FP64 and FX64 with a
roofline for each sweep kernel and the FP32-vs-FP64 accuracy contract; the
256 ragged jobs as one graph-captured batch; the serving trace (24 requests x
5000 sweeps under a binding field-memory budget) beside the plain FP64
per-job path on the same shapes; and the paper's benchmark protocol at two
chain lengths against one host core.

--impl reference times the CPU oracle (plain C, FP64, local-field mode) on
the host cores on a bounded sample of the same workload.
Under torchrun (N > 1) every rank runs its own eight chains (seeds offset by
8 x rank): the chains are independent, so the work shards with no data-path
collective and the scaling is weak.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SWEEPS_PER_STEP = 10
L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="chains", choices=["chains", "precision", "batching", "serving", "paper"])
    ap.add_argument("--serve-jobs", type=int, default=24)
    ap.add_argument("--serve-sweeps", type=int, default=5000)
    ap.add_argument("--serve-budget-mib", type=float, default=64.0)
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-precision", action="store_true")
    ap.add_argument("--no-batching", action="store_true")
    ap.add_argument("--no-paper", action="store_true")
    ap.add_argument("--precision", default=None, choices=[None, "fp64", "fp32", "fx64"])
    ap.add_argument("--no-fp32-compare", action="store_true")
    ap.add_argument("--no-fx64-compare", action="store_true")
    ap.add_argument("--no-direct-compare", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    return ap.parse_args()


def rank_max(x, world, device):
    """The largest x over the ranks (the job's time is its slowest rank's)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_min(x, world, device):
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MIN)
    return float(t.item())


def job_rate(total_attempts, slowest_ms):
    """Whole-job attempts/s: the attempts of all ranks over the slowest rank's time."""
    return total_attempts / (slowest_ms / 1e3)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload_specs(name, rank, precision):
    from paper_1308_5426_gb300 import workloads
    if name == "chains":
        specs = workloads.chains_jobs()
        for s in specs:
            s.seed += 8 * rank
            s.precision = precision or "fp64"
        desc = {"workload": "8 independent PT chains, L=1024 q=5 sigma=0.4 R=64, T/Jtot geometric 0.05-1, "
                            "exchange every sweep, E/M every 10 sweeps",
                "L": 1024, "q": 5, "sigma": 0.4, "R": 64, "chains": 8}
    elif name == "precision":
        s = workloads.precision_job(precision or "fp32")
        s.seed += rank
        specs = [s]
        desc = {"workload": "one PT job, L=4096 q=8 sigma=0.2 R=128, T/Jtot geometric 0.02-0.5, "
                            "exchange every sweep, E/M every 10 sweeps, FP32 rebuild every 100 sweeps",
                "L": 4096, "q": 8, "sigma": 0.2, "R": 128, "chains": 1}
    elif name == "batching":
        specs = workloads.batching_jobs()
        desc = {"workload": "256 ragged PT jobs (L 256-8192, q 2-10, sigma U[0.1,1], R 32/64/128, FP32, "
                            "rebuild every 100 sweeps) in one graph-captured batch; step = 1 sweep + exchange",
                "jobs": 256}
    elif name == "paper":
        specs = workloads.paper_benchmark_jobs()
        desc = {"workload": "the paper's benchmark protocol (Sec. 5.2): q=3, sigma=0.2, 400 replicas on a "
                            "uniform temperature grid, L=512..10240, production sweeps 1e4 (L=512) down to 50 "
                            "(L=10240) + 20% thermalisation, from random spins; plus the replica scan of Fig. 5 "
                            "(L=1024)"}
    else:
        specs = workloads.serving_trace()[:1]
        desc = {"workload": "serving trace: Poisson(50/s) arrivals, q 3/5/8, sigma U[0.1,1], L 512-16384, "
                            "R=64, FP32, continuous batching"}
    return specs, desc


# ----------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------- peaks
def peaks():
    p = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
    except (OSError, ValueError):
        pass
    return p


SWEEP_SOURCES = ["sweep.cu", "sweep_common.cuh", "near_tie.cuh", "sweep_sched.cuh", "philox.cuh", "potts_internal.h"]
SWEEP_PROFILE = os.path.join(ROOT, "profiles", "sweep_fp64_chains_L1024_q5.md")


def profiled_traffic():
    """DRAM bytes per launch of the FP64 sweep kernel from its committed ncu
    summary, or None if the kernel sources changed since the capture."""
    import hashlib
    try:
        h = hashlib.sha256()
        for f in SWEEP_SOURCES:
            with open(os.path.join(ROOT, "paper_1308_5426_gb300", "csrc", f), "rb") as fh:
                h.update(fh.read())
        digest = h.hexdigest()[:16]
        vals = {}
        with open(SWEEP_PROFILE) as fh:
            for line in fh:
                parts = line.strip().split(":")
                if len(parts) == 2 and parts[0] in ("source_sha256_16", "traffic_bytes_per_launch"):
                    vals[parts[0]] = parts[1].strip()
        if vals.get("source_sha256_16") == digest:
            return int(vals["traffic_bytes_per_launch"])
    except (OSError, ValueError, KeyError):
        pass
    return None


# shared-memory (or L2) bytes of one FX64 field update (one element of one
# accepted flip): the two 8-byte field words read and written, the 8-byte
# coupling read
FX64_BYTES_PER_UPDATE = 5 * 8

KERNEL_NAMES = {"memory": "sweep_kernel", "registers": "sweep_rf_kernel", "cluster": "sweep_cluster_kernel",
                "direct": "sweep_direct_kernel"}


FIELD_TYPE = {"fp64": "double", "fp32": "float", "fx64": "long long"}
FIELD_NAME = {"fp64": "FP64", "fp32": "FP32", "fx64": "FX64"}


def kernel_label(info, prec):
    """Name of the sweep kernel a job ran, from the library's own report
    (potts_lr_sweep_info), with where its fields and table live."""
    k = info["kernel"]
    if k == "memory":
        where = "fields %s, table %s" % ("in shared memory" if info["fields_in_smem"] else "in global memory",
                                         "in shared memory" if info["table_in_smem"] else "in global memory")
        return "sweep_kernel<%s> (%s)" % (FIELD_TYPE[prec], where)
    if k == "registers":
        return "sweep_rf_kernel<%s> (%s fields in registers, configuration %d)" % (
            FIELD_TYPE[prec], FIELD_NAME[prec], info["register_config"])
    if k == "cluster":
        return "sweep_cluster_kernel<%s> (%s fields shared by a %d-CTA cluster)" % (
            FIELD_TYPE[prec], FIELD_NAME[prec], info["cluster"])
    if k == "register_cluster":
        return "sweep_rfc_kernel<%s> (%s fields in the registers of a %d-CTA cluster)" % (
            FIELD_TYPE[prec], FIELD_NAME[prec], info["cluster"])
    return "sweep_direct_kernel (no fields)"


def sweep_roofline(plr, res, specs, sm_max_mhz, nsms):
    """Roofline entry of the sweep kernel of a timed_device run.  Work per
    attempt: A * 2L field additions (FP64 and FP32: against the add pipe's
    unit-count peak and its measured probe); FX64: A * L element updates of
    40 bytes against the measured shared-memory probe where the fields sit in
    shared memory (one CTA or a cluster), the measured L2 probe where they
    sit in global memory, and for fields in registers A * 2L 64-bit integer
    adds against the measured integer-add probe.  A = the measured
    acceptance; achieved = the work of one launch over the average sweep
    launch time (CUDA events on the launching stream)."""
    info = res["info"]
    prec = specs[0].precision
    A = res["acceptance"]
    att_launch = sum(s.L * s.R for s in specs)
    upd_launch = sum(s.L * s.R * s.L for s in specs) * A  # element updates per launch (per state row pair)
    sweep_s = float(np.mean(res["sweep_ms"])) / 1e3
    kernel = kernel_label(info, prec)
    if prec == "fx64" and info["kernel"] in ("registers", "register_cluster"):
        peak = plr.probe("i64_add")
        achieved = 2.0 * upd_launch / sweep_s
        roof = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "Tadd/s",
                "frac": achieved / peak, "traffic": None, "kernel": kernel,
                "work": "A*2L 64-bit integer adds per attempt (two field words per element), A=%.4f measured; "
                        "%d attempts per launch" % (A, att_launch),
                "peak_source": "measured 64-bit integer add probe (potts_lr_probe)", "sweep_ms_avg": sweep_s * 1e3}
    elif prec == "fx64":
        where = "smem" if (info["fields_in_smem"] or info["kernel"] == "cluster") else "l2"
        peak = plr.probe(where)
        achieved = upd_launch * FX64_BYTES_PER_UPDATE / sweep_s
        roof = {"bound": where, "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "GB/s",
                "frac": achieved / peak, "traffic": None, "kernel": kernel,
                "work": "A*L element updates per attempt, %d bytes each, A=%.4f measured; %d attempts per launch"
                        % (FX64_BYTES_PER_UPDATE, A, att_launch),
                "peak_source": "measured %s probe (potts_lr_probe)" % ("shared-memory" if where == "smem" else "L2"),
                "sweep_ms_avg": sweep_s * 1e3}
    else:
        kind = "fp32" if prec == "fp32" else "fp64"
        peak = alu_peak(kind, sm_max_mhz)
        achieved = 2.0 * upd_launch / sweep_s
        measured = plr.probe(kind + "_add")
        roof = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None,
                "peak_measured_probe": measured / 1e12, "frac_of_measured_probe": achieved / measured,
                "kernel": kernel,
                "work": "A*2L %s adds per attempt, A=%.4f measured; %d attempts per launch" % (prec, A, att_launch),
                "peak_source": "unit counts x max SM clock (2 FP64 / 128 FP32 add lanes per SM per clock, 152 SMs)",
                "sweep_ms_avg": sweep_s * 1e3}
    nslots = sum(s.R for s in specs)
    if nslots < nsms and info["kernel"] not in ("cluster", "register_cluster"):  # also against the occupied SMs
        roof["frac_of_occupied_sms"] = roof["frac"] * nsms / nslots
        roof["occupied_sms"] = nslots
    if prec == "fp32":
        roof["sweep_ms_note"] = ("the timed sweep includes the conditional rebuild launches that follow every FP32 "
                                 "sweep (they exit at once unless a rebuild is due)")
    return roof


def alu_peak(kind, sm_max_mhz):
    """ALU peaks from unit counts and the maximum SM clock: 152 SMs; FP32: 128
    lanes/clk/SM; FP64: the nominal 1.25 TFLOP/s of GB300 is 2 FMA/clk/SM at
    2070 MHz, i.e. 2 FP64 adds/clk/SM."""
    f = (sm_max_mhz or 2070.0) * 1e6
    lanes = {"fp64": 2.0, "fp32": 128.0}[kind]
    return 152 * lanes * f  # adds per second


# ----------------------------------------------------------------- CPU baseline
def cpu_baseline(specs, seconds):
    """The oracle as it stands (local-field mode, FP64), one replica per POSIX
    thread over all host cores, on a bounded sample: the first chain, as many
    sweeps as fit in about `seconds`."""
    import oracle
    s = specs[0]
    temps = s.ratios * oracle.jtot(s.L, s.sigma)
    cores = os.cpu_count() or 1
    o = oracle.Oracle(s.L, s.q, s.sigma, temps, s.seed)
    t0 = time.perf_counter()
    o.step(mode="field", nthreads=cores)
    t1 = time.perf_counter()
    per = max(t1 - t0, 1e-4)
    n = max(1, min(2000, int(seconds / per)))
    t0 = time.perf_counter()
    for _ in range(n):
        o.step(mode="field", nthreads=cores)
    dt = time.perf_counter() - t0
    att = n * s.L * s.R
    # one core, as the paper compares with (Sec. 5.2): the same chain, about a
    # third of the time budget
    t0 = time.perf_counter()
    o.step(mode="field", nthreads=1)
    per1 = max(time.perf_counter() - t0, 1e-4)
    n1 = max(1, min(500, int(seconds / 3 / per1)))
    t0 = time.perf_counter()
    for _ in range(n1):
        o.step(mode="field", nthreads=1)
    dt1 = time.perf_counter() - t0
    return {"value": att / dt, "unit": "attempts/s", "cores": cores, "kind": "oracle",
            "sample": "chain 1 of the workload (L=%d q=%d R=%d), %d sweeps + exchanges, FP64 local-field "
                      "mode, %.1f s" % (s.L, s.q, s.R, n, dt),
            "one_core": {"value": n1 * s.L * s.R / dt1, "unit": "attempts/s", "cores": 1,
                         "sample": "the same chain, %d sweeps + exchanges on one thread, %.1f s" % (n1, dt1)}}


def run_reference(args, specs, desc, rank, world):
    """--impl reference: the CPU oracle, K steps, each a bounded sample."""
    if rank != 0:
        return 0
    import oracle
    s = specs[0]
    temps = s.ratios * oracle.jtot(s.L, s.sigma)
    cores = os.cpu_count() or 1
    o = oracle.Oracle(s.L, s.q, s.sigma, temps, s.seed)
    for _ in range(args.warmup):
        o.step(mode="field", nthreads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step(mode="field", nthreads=cores)
    dt = time.perf_counter() - t0
    att = args.steps * s.L * s.R
    v = att / dt
    line = {"impl": "reference", "metric": "spin-flip attempts/s", "value": v, "unit": "attempts/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": desc,
            "cpu_baseline": {"value": v, "unit": "attempts/s", "cores": cores, "kind": "oracle",
                             "sample": "each step: one sweep + exchange of chain 1 (L=%d q=%d R=%d), FP64 "
                                       "local-field mode, %d threads" % (s.L, s.q, s.R, cores)},
            "e2e": {"value": v, "unit": "attempts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- GPU arm
def make_jobs(plr, specs, stream, variant="auto", site_order="sequential"):
    return [plr.Job(s.L, s.q, s.sigma, s.ratios * plr.jtot(s.L, s.sigma), s.seed, precision=s.precision,
                    stream=stream, sweep_variant=variant, site_order=site_order) for s in specs]


def timed_device(plr, torch, specs, steps, warmup, dev, with_events=True, variant="auto", site_order="sequential"):
    st = torch.cuda.Stream(device=dev)
    jobs = make_jobs(plr, specs, st.cuda_stream, variant, site_order)
    batch = plr.Batch(jobs, stream=st.cuda_stream)
    nslots = batch.nslots
    Eb = torch.empty(nslots, dtype=torch.float64, device=dev)
    Mb = torch.empty(nslots, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    att_step = SWEEPS_PER_STEP * sum(s.L * s.R for s in specs)

    def step(sweep_ev=None):
        for _ in range(SWEEPS_PER_STEP):
            if sweep_ev is not None:
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(st)
                batch.sweep(1)
                b.record(st)
                sweep_ev.append((a, b))
            else:
                batch.sweep(1)
            batch.exchange()
        batch.measure_device(Eb.data_ptr(), Mb.data_ptr())

    for _ in range(warmup):
        step()
    batch.sync()
    acc0 = sum(int(j.stats()["acc_flip"].sum()) for j in jobs)
    step_ev, sweep_ev = [], []
    torch.cuda.synchronize(dev)
    for _ in range(steps):
        with torch.cuda.stream(st):
            flush.zero_()  # L2 flush between timed steps, outside the step's events
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        step(sweep_ev if with_events else None)
        b.record(st)
        step_ev.append((a, b))
    torch.cuda.synchronize(dev)
    acc1 = sum(int(j.stats()["acc_flip"].sum()) for j in jobs)
    step_ms = sum(a.elapsed_time(b) for a, b in step_ev)
    sweep_ms = [a.elapsed_time(b) for a, b in sweep_ev]
    out = {"step_ms": step_ms, "att_step": att_step, "acceptance": (acc1 - acc0) / (steps * att_step),
           "sweep_ms": sweep_ms, "steps": steps, "info": jobs[0].sweep_info()}
    batch.close()
    for j in jobs:
        j.close()
    return out


def timed_e2e(plr, torch, specs, steps, warmup, dev):
    """Through the public API with host buffers: each step restores every
    chain from a pinned host checkpoint (H2D, one batch call), runs 10 sweeps +
    exchanges, measures into host arrays (D2H) and checkpoints every chain back
    (D2H, one batch call)."""
    st = torch.cuda.Stream(device=dev)
    jobs = make_jobs(plr, specs, st.cuda_stream)
    batch = plr.Batch(jobs, stream=st.cuda_stream)
    size = batch.state_size()  # every chain's checkpoint, back to back
    buf = torch.empty(size, dtype=torch.uint8, pin_memory=True)
    batch.get_state_into(buf.data_ptr(), size)
    E = np.zeros(batch.nslots)
    M = np.zeros(batch.nslots)
    att_step = SWEEPS_PER_STEP * sum(s.L * s.R for s in specs)

    def step():
        batch.set_state_from(buf.data_ptr(), size)
        batch.run(SWEEPS_PER_STEP, SWEEPS_PER_STEP)
        E[:], M[:] = batch.measure()
        batch.get_state_into(buf.data_ptr(), size)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(steps):
        step()
    torch.cuda.synchronize(dev)
    dt = time.perf_counter() - t0
    h2d = size
    d2h = size + 2 * 8 * batch.nslots
    batch.close()
    for j in jobs:
        j.close()
    return {"value": steps * att_step / dt, "unit": "attempts/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h}


def per_job_rates(plr, torch, dev, reqs, precision, min_seconds=0.25, max_sweeps=200, warm_sweeps=30,
                  warm_seconds=1.0):
    """Each request's shape as a plain job of the given precision, alone on the
    GPU (the per-job path), from its random start: warm-up sweeps + exchanges
    past the quench from random spins (warm_sweeps, or fewer where they would
    take more than about warm_seconds), then as many timed sweeps + exchanges
    as take about min_seconds (CUDA events on the job's stream, at least two).
    Returns the attempts a request asks for, the time the per-job path needs
    for all of them at its sampled rate, and the samples."""
    st = torch.cuda.Stream(device=dev)
    total_att, total_s, rows = 0, 0.0, []
    for r in reqs:
        j = plr.Job(r.L, r.q, r.sigma, r.temps, r.seed, precision=precision, stream=st.cuda_stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        j.sweep(1)
        j.exchange()
        e1.record(st)
        e1.synchronize()
        first = max(e0.elapsed_time(e1) / 1e3, 1e-6)
        nwarm = max(0, min(warm_sweeps, int(warm_seconds / first)) - 1)
        e0.record(st)
        for _ in range(nwarm):
            j.sweep(1)
            j.exchange()
        e1.record(st)
        e1.synchronize()
        if nwarm:
            first = max(e0.elapsed_time(e1) / 1e3 / nwarm, 1e-6)
        n = max(2, min(max_sweeps, int(min_seconds / first)))
        e0.record(st)
        for _ in range(n):
            j.sweep(1)
            j.exchange()
        e1.record(st)
        e1.synchronize()
        dt = e0.elapsed_time(e1) / 1e3
        rate = n * r.L * r.R / dt
        rows.append({"L": r.L, "q": r.q, "sigma": round(r.sigma, 4), "warm_sweeps": nwarm + 1, "sampled_sweeps": n,
                     "attempts_per_s": rate,
                     "kernel": kernel_label(j.sweep_info(), precision)})
        total_att += r.attempts
        total_s += r.attempts / rate
        j.close()
    return total_att, total_s, rows


def rebuild_shares(plr, torch, dev, reqs, min_L=4096):
    """Share of the FP32 step time spent in the tensor-core rebuilds and
    energy re-anchors, per served shape with L >= min_L: the same job alone,
    20 sweeps + exchanges timed (CUDA events) after its schedule settled,
    with the adaptive rebuild (K = 100) and with none (K = 0)."""
    out = []
    for L, q, sigma in sorted({(r.L, r.q, r.sigma) for r in reqs if r.L >= min_L}):
        ms = {}
        for K in (0, 100):
            st = torch.cuda.Stream(device=dev)
            temps = [r for r in reqs if (r.L, r.q, r.sigma) == (L, q, sigma)][0].temps
            j = plr.Job(L, q, sigma, temps, 5, precision="fp32", recompute_every=K, stream=st.cuda_stream)
            for _ in range(60 if L >= 16384 else 150):
                j.sweep(1)
                j.exchange()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(20):
                j.sweep(1)
                j.exchange()
            e1.record(st)
            e1.synchronize()
            ms[K] = e0.elapsed_time(e1) / 20
            if K:
                info = j.rebuild_info()
            j.close()
        out.append({"L": L, "q": q, "sigma": round(sigma, 4), "ms_per_step_no_rebuild": ms[0],
                    "ms_per_step_adaptive": ms[100], "rebuild_share": 1.0 - ms[0] / ms[100],
                    "settled_interval": info["interval"], "last_drift": info["last_drift"]})
    return out


def serving_run(plr, torch, dev, njobs, sweeps, budget_bytes):
    """The serving trace (Poisson arrivals at 50 jobs/s; q in {3,5,8}, sigma in
    U[0.1,1], L in {512..16384}, R=64, FP32 fields, K=100) cut to its first
    njobs requests, each with its stated `sweeps`, served with continuous
    batching on the wall clock under a field-memory budget (L q R 4 bytes per
    job) small enough that admission binds.  Then the same requests, every one
    of them, on the plain FP64 per-job path (and the exact FX64 one): each
    shape alone on the GPU, its rate sampled, and the time the whole request
    would take at that rate -- equal work on both sides of the ratio."""
    from paper_1308_5426_gb300 import workloads
    from paper_1308_5426_gb300.serve import GpuEngine, Request, Server

    trace = workloads.serving_trace()[:njobs]
    reqs = []
    for i, sp in enumerate(trace):
        temps = sp.ratios * plr.jtot(sp.L, sp.sigma)
        reqs.append(Request(rid=i, L=sp.L, q=sp.q, sigma=sp.sigma, temps=temps, seed=sp.seed, sweeps=sweeps,
                            recompute_every=100, arrival=sp.arrival))

    rebuilds = {}

    class Engine(GpuEngine):
        """The library's engine, recording each finished job's field error and
        rebuild schedule."""
        max_err = 0.0
        peak_used = 0

        def destroy(self, job):
            Engine.max_err = max(Engine.max_err, job.fields_error())
            rebuilds.setdefault((job.L, job.q), []).append(job.rebuild_info())
            job.close()

    st = torch.cuda.Stream(device=dev)
    srv = Server(Engine(stream=st.cuda_stream), budget_bytes=budget_bytes, chunk=10)
    max_concurrent = [0]
    orig_admit = srv._admit

    def admit(now):
        ok = orig_admit(now)
        max_concurrent[0] = max(max_concurrent[0], len(srv.active))
        Engine.peak_used = max(Engine.peak_used, srv.used)
        return ok
    srv._admit = admit
    t0 = time.perf_counter()
    srv.run(reqs, idle_sleep=1e-4)
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - t0
    summ = srv.summary(wall_seconds=wall)
    waited = [r.admitted - r.arrival for r in srv.results.values() if r.admitted is not None]
    shares = rebuild_shares(plr, torch, dev, reqs)
    att64, t64, rows64 = per_job_rates(plr, torch, dev, reqs, "fp64")
    attx, tx, rowsx = per_job_rates(plr, torch, dev, reqs, "fx64")
    served = summ.get("attempts_per_s") or 0.0
    return {"jobs": len(reqs), "sweeps_per_job": sweeps,
            "trace": "first %d requests of the 500-request Poisson(50/s) trace, seed 5, each with its stated "
                     "%d sweeps" % (len(reqs), sweeps),
            "budget_bytes": budget_bytes, "total_footprint_bytes": sum(r.footprint for r in reqs),
            "peak_admitted_bytes": Engine.peak_used, "max_concurrent_jobs": max_concurrent[0],
            "max_queue_wait_s": max(waited) if waited else None,
            "wall_s": wall, "attempts": summ["attempts"], "attempts_per_s": served,
            "attempts_per_busy_s": summ.get("attempts_per_busy_s"),
            "p50_latency_s": summ.get("p50_s"), "p99_latency_s": summ.get("p99_s"), "done": summ["done"],
            "max_field_error_rel_jtot": Engine.max_err,
            "rebuild_by_shape": [{"L": L, "q": q, "settled_interval": [r["interval"] for r in v],
                                  "rebuilds_per_job": [r["rebuilds"] for r in v]}
                                 for (L, q), v in sorted(rebuilds.items())],
            "rebuild_share_by_shape": shares,
            "fp64_per_job_attempts_per_s": att64 / t64,
            "fp64_per_job": "every request's shape as a plain FP64 job alone on the GPU, rate sampled over >= 0.25 s "
                            "after up to 30 warm-up sweeps (about 1 s at most) from random spins; the full %d sweeps "
                            "of all %d requests would take %.0f s at those rates" % (sweeps, len(reqs), t64),
            "fp64_per_job_samples": rows64,
            "fx64_per_job_attempts_per_s": attx / tx, "fx64_per_job_samples": rowsx,
            "served_fp32_over_fp64_per_job": served / (att64 / t64),
            "served_fp32_over_fx64_per_job": served / (attx / tx)}


def batching_run(plr, torch, dev, steps, warmup, sm_max_mhz=None):
    """The 256 ragged jobs (L in {256..8192}, q in 2..10, sigma in U[0.1,1],
    R in {32,64,128}, FP32, K=100) created together and stepped as one
    graph-captured batch; each step = one sweep of every slot of every job +
    one exchange step per job (+ the rebuilds that fall due).  The roofline
    is that of the whole step: the FP32 field additions of every accepted flip
    (2L per flip, counted from each job's own acceptance counters) over the
    step time, against the FP32 add pipe's unit-count peak."""
    from paper_1308_5426_gb300 import workloads
    specs = workloads.batching_jobs()
    st = torch.cuda.Stream(device=dev)
    jobs = make_jobs(plr, specs, st.cuda_stream)
    b = plr.Batch(jobs, stream=st.cuda_stream)
    b.run(warmup, max(1, warmup))
    b.sync()
    acc0 = [int(j.stats()["acc_flip"].sum()) for j in jobs]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    b.run(steps, min(10, steps))
    e1.record(st)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    acc1 = [int(j.stats()["acc_flip"].sum()) for j in jobs]
    att = steps * sum(s.L * s.R for s in specs)
    adds = sum(2.0 * s.L * (a1 - a0) for s, a0, a1 in zip(specs, acc0, acc1))
    kinds = {}
    for j in jobs:
        k = j.sweep_info()["kernel"]
        kinds[k] = kinds.get(k, 0) + 1
    b.close()
    for j in jobs:
        j.close()
    peak = alu_peak("fp32", sm_max_mhz)
    achieved = adds / (ms / 1e3)
    return {"jobs": len(specs), "slots": sum(s.R for s in specs), "steps": steps, "ms": ms,
            "attempts_per_s": att / (ms / 1e3), "unit": "attempts/s",
            "acceptance": sum(a1 - a0 for a0, a1 in zip(acc0, acc1)) / att, "sweep_kernels": kinds,
            "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None,
                         "kernel": "the whole batch step (every sweep kernel, rebuilds, exchanges)",
                         "work": "2L FP32 adds per accepted flip, summed over the jobs' own counters",
                         "peak_source": "unit counts x max SM clock (128 FP32 add lanes per SM per clock, 152 SMs)"}}


def precision_legs(plr, torch, dev, steps, warmup, sm_max_mhz, nsms):
    """The precision job (L=4096 q=8 sigma=0.2 R=128, T/Jtot geometric
    0.02-0.5, seed 1) in FP32 (split-BF16 tensor-core rebuilds, K=100), plain
    FP64 and FX64 fields: each timed alone (step = 10 sweeps + exchanges + one
    measurement), with the roofline of its sweep kernel."""
    from paper_1308_5426_gb300 import workloads
    out = {}
    for prec in ("fp32", "fp64", "fx64"):
        spec = workloads.precision_job(prec)
        r = timed_device(plr, torch, [spec], steps, warmup, dev)
        out["precision_" + prec] = {"value": r["steps"] * r["att_step"] / (r["step_ms"] / 1e3),
                                    "unit": "attempts/s", "acceptance": r["acceptance"],
                                    "ms_per_step": r["step_ms"] / r["steps"],
                                    "roofline": sweep_roofline(plr, r, [spec], sm_max_mhz, nsms)}
    return out


def precision_accuracy(plr, torch, dev, warm=500, prod=2000, nbins=20, check_every=10):
    """The precision contract on the precision job, same seed and call
    sequence in FP32 (K=100) and FP64: the FP32 field drift (max |h32 - h64| /
    Jtot, h64 the FP64 direct sums of the same spins) at a check every 10
    sweeps over the whole run, and after `warm` sweeps the difference of <E>/L
    and <M> per slot over `prod` sweeps (measured every sweep on the device,
    binned in `nbins` bins) in units of the combined binned standard error."""
    import math
    from paper_1308_5426_gb300 import workloads
    data, drift = {}, []
    for prec in ("fp32", "fp64"):
        spec = workloads.precision_job(prec)
        st = torch.cuda.Stream(device=dev)
        j = make_jobs(plr, [spec], st.cuda_stream)[0]
        Eb = torch.zeros((prod, spec.R), dtype=torch.float64, device=dev)
        Mb = torch.zeros((prod, spec.R), dtype=torch.float64, device=dev)
        for n in range(warm + prod):
            j.sweep(1)
            j.exchange()
            if n >= warm:
                j.measure_device(Eb[n - warm].data_ptr(), Mb[n - warm].data_ptr())
            if prec == "fp32" and (n + 1) % check_every == 0:
                drift.append(j.fields_error())
        j.sync()
        data[prec] = ((Eb / spec.L).cpu().numpy(), Mb.cpu().numpy())
        j.close()
    out = {"protocol": "L=4096 q=8 sigma=0.2 R=128, seed 1, FP32 (K=100) vs FP64; %d warm-up + %d measured "
                       "sweeps (each followed by an exchange), %d bins; drift checked every %d sweeps"
                       % (warm, prod, nbins, check_every),
           "max_field_drift_rel_jtot": max(drift), "drift_checks": len(drift)}
    for k, name in ((0, "E_per_site"), (1, "M")):
        stats = []
        for prec in ("fp32", "fp64"):
            x = data[prec][k]
            b = x[: (x.shape[0] // nbins) * nbins].reshape(nbins, -1, x.shape[1]).mean(axis=1)
            stats.append((b.mean(axis=0), b.std(axis=0, ddof=1) / math.sqrt(nbins)))
        (m32, s32), (m64, s64) = stats
        se = np.hypot(s32, s64)
        diff = m32 - m64
        frozen = se <= 1e-12 * np.maximum(np.abs(m64), 1.0)
        z = np.where(frozen, 0.0, diff / np.where(frozen, 1.0, se))
        out[name] = {"max_abs_fp32_minus_fp64": float(np.abs(diff).max()),
                     "max_abs_diff_over_se": float(np.abs(z).max()),
                     "slots_beyond_3_se": int((np.abs(diff) >= 3 * se + 1e-12).sum()),
                     "frozen_slots_equal": bool(np.all(diff[frozen] == 0)), "frozen_slots": int(frozen.sum())}
    return out


def paper_run(plr, torch, dev, seconds_per_case=2.0, Ls=None, scan=True):
    """The paper's benchmark (Sec. 5.2, Fig. 4) and replica scan (Fig. 5) on
    this GPU, FP32 and FP64, against the oracle on one host core.  Each GPU
    case runs the protocol's sweeps from random spins (cut to about
    seconds_per_case); the oracle runs 8 of the 400 temperatures (every 50th)
    from random spins for as many sweeps as fit in about seconds_per_case.
    Ls: the chain lengths to run (default all nine); scan: the replica scan."""
    import oracle
    from paper_1308_5426_gb300 import workloads

    def gpu_rate(s, R, precision, sweeps):
        temps = workloads.uniform_ratios(R, 0.1, 1.0) * plr.jtot(s.L, s.sigma)
        st = torch.cuda.Stream(device=dev)
        j = plr.Job(s.L, s.q, s.sigma, temps, s.seed, precision=precision, stream=st.cuda_stream)
        j.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        j.sweep(1)
        j.exchange()
        e1.record(st)
        e1.synchronize()
        first = max(e0.elapsed_time(e1) / 1e3, 1e-6)
        n = max(1, min(sweeps - 1, int(seconds_per_case / first)))
        e0.record(st)
        for _ in range(n):
            j.sweep(1)
            j.exchange()
        e1.record(st)
        e1.synchronize()
        dt = e0.elapsed_time(e1) / 1e3
        j.close()
        return n * s.L * R / dt, n + 1

    def cpu_rate(s):
        temps = workloads.uniform_ratios(400, 0.1, 1.0)[::50] * oracle.jtot(s.L, s.sigma)
        o = oracle.Oracle(s.L, s.q, s.sigma, temps, s.seed)
        t0 = time.perf_counter()
        n = 0
        while n < s.sweeps and (n == 0 or time.perf_counter() - t0 < seconds_per_case):
            o.step(mode="field", nthreads=1)
            n += 1
        dt = time.perf_counter() - t0
        return n * s.L * len(temps) / dt, n

    table = []
    for s in workloads.paper_benchmark_jobs():
        if Ls is not None and s.L not in Ls:
            continue
        g32, n32 = gpu_rate(s, 400, "fp32", s.sweeps)
        g64, n64 = gpu_rate(s, 400, "fp64", s.sweeps)
        c1, nc = cpu_rate(s)
        table.append({"L": s.L, "R": 400, "protocol_sweeps": s.sweeps, "gpu_fp32": g32, "gpu_fp32_sweeps": n32,
                      "gpu_fp64": g64, "gpu_fp64_sweeps": n64, "oracle_1core": c1, "oracle_sweeps": nc,
                      "speedup_fp32_vs_1core": g32 / c1, "speedup_fp64_vs_1core": g64 / c1})
    if not scan:
        return {"fig4_table": table,
                "oracle_sample": "8 of the 400 temperatures (every 50th), one thread, FP64 local-field mode, "
                                 "from random spins"}
    s1024 = [s for s in workloads.paper_benchmark_jobs() if s.L == 1024][0]
    c1024 = [row["oracle_1core"] for row in table if row["L"] == 1024][0]
    scan = []
    for R in (112, 224, 336, 448, 560):
        g, n = gpu_rate(s1024, R, "fp32", s1024.sweeps)
        scan.append({"L": 1024, "R": R, "gpu_fp32": g, "sweeps": n, "speedup_fp32_vs_1core": g / c1024})
    return {"fig4_table": table, "fig5_replica_scan": scan,
            "oracle_sample": "8 of the 400 temperatures (every 50th), one thread, FP64 local-field mode, "
                             "from random spins"}


def main():
    args = parse()
    rank, world, local = dist_env()
    specs, desc = workload_specs(args.workload, rank, args.precision)
    if args.impl == "reference":
        return run_reference(args, specs, desc, rank, world)

    import torch
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    import paper_1308_5426_gb300 as plr
    from paper_1308_5426_gb300 import _lib
    _lib.load()

    clocks = ClockSampler(local)
    if args.workload == "paper":
        if rank != 0:
            return 0
        torch.cuda.synchronize(dev)
        clocks.start()
        r = paper_run(plr, torch, dev)
        ck = clocks.stop()
        tot = sum(row["gpu_fp32"] for row in r["fig4_table"]) / len(r["fig4_table"])
        line = {"metric": "spin-flip attempts/s", "value": tot, "unit": "attempts/s", "n_gpus": 1,
                "steps": len(r["fig4_table"]), "warmup": 0, "ms_per_step": None, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": desc,
                "clocks": ck, "value_is": "mean over the Fig. 4 lengths of the FP32 attempts/s",
                "detail": r, "roofline": None, "e2e": None, "cpu_baseline": None}
        print(json.dumps(line), flush=True)
        return 0
    if args.workload in ("batching", "serving"):
        torch.cuda.synchronize(dev)
        clocks.start()
        if args.workload == "batching":
            r = batching_run(plr, torch, dev, args.steps, args.warmup)
            value, ms_step = r["attempts_per_s"], r["ms"] / args.steps
        else:
            r = serving_run(plr, torch, dev, args.serve_jobs, args.serve_sweeps,
                            int(args.serve_budget_mib * 2 ** 20))
            value, ms_step = r["attempts_per_s"], 1e3 * r["wall_s"]
        ck = clocks.stop()
        if rank == 0:
            line = {"metric": "spin-flip attempts/s", "value": value, "unit": "attempts/s", "n_gpus": world,
                    "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
                    "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                    "config": desc, "clocks": ck, "detail": r, "roofline": None, "e2e": None,
                    "cpu_baseline": None}
            print(json.dumps(line), flush=True)
        return 0
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    res = timed_device(plr, torch, specs, args.steps, args.warmup, dev)
    ck = clocks.stop()
    step_ms = rank_max(res["step_ms"], world, dev)
    value = job_rate(world * args.steps * res["att_step"], step_ms)

    # roofline of the sweep kernel (the dominant kernel)
    prec = specs[0].precision
    A = res["acceptance"]
    nsms = torch.cuda.get_device_properties(dev).multi_processor_count
    roof = sweep_roofline(plr, res, specs, ck.get("sm_max_mhz"), nsms)
    if args.workload == "chains" and prec == "fp64":
        roof["traffic"] = profiled_traffic()

    extra = {}
    if args.workload == "chains" and not args.no_fp32_compare and prec == "fp64":
        specs32, _ = workload_specs(args.workload, rank, "fp32")
        r32 = timed_device(plr, torch, specs32, max(3, args.steps // 3), args.warmup, dev)
        extra["fp32_same_workload"] = {"value": world * r32["steps"] * r32["att_step"] / (r32["step_ms"] / 1e3),
                                       "unit": "attempts/s", "acceptance": r32["acceptance"],
                                       "roofline": sweep_roofline(plr, r32, specs32, ck.get("sm_max_mhz"), nsms)}
    if args.workload == "chains" and not args.no_fx64_compare and prec == "fp64":
        # the same chains with 64-bit fixed-point fields: exact integer updates,
        # the same FP64 decisions
        specsx, _ = workload_specs(args.workload, rank, "fx64")
        rx = timed_device(plr, torch, specsx, max(3, args.steps // 3), args.warmup, dev)
        extra["fx64_same_workload"] = {
            "value": world * rx["steps"] * rx["att_step"] / (rx["step_ms"] / 1e3), "unit": "attempts/s",
            "acceptance": rx["acceptance"], "roofline": sweep_roofline(plr, rx, specsx, ck.get("sm_max_mhz"), nsms)}
    if args.workload == "chains" and not args.no_direct_compare and prec == "fp64":
        # the paper's scheme on the same workload: every proposal sums its O(L)
        # interaction (no fields), FP64
        rd = timed_device(plr, torch, specs, max(3, args.steps // 10), args.warmup, dev, with_events=False,
                          variant="direct")
        extra["fp64_direct_same_workload"] = {
            "value": world * rd["steps"] * rd["att_step"] / (rd["step_ms"] / 1e3), "unit": "attempts/s",
            "acceptance": rd["acceptance"],
            "kernel": "sweep_direct_kernel: the paper's O(L)-per-attempt sum, no local fields (Sec. 4.2)"}
        rr = timed_device(plr, torch, specs, max(3, args.steps // 10), args.warmup, dev, with_events=False,
                          site_order="random")
        extra["fp64_random_sites_same_workload"] = {
            "value": world * rr["steps"] * rr["att_step"] / (rr["step_ms"] / 1e3), "unit": "attempts/s",
            "acceptance": rr["acceptance"],
            "kernel": "sweep_direct_kernel with random site order (attempts at Philox-drawn sites)"}

    if args.workload == "chains" and world == 1:
        # the other workloads of the contract, each timed on its own stream
        if not args.no_precision:
            extra.update(precision_legs(plr, torch, dev, max(3, args.steps // 4), max(3, args.warmup),
                                        ck.get("sm_max_mhz"), nsms))
            extra["precision_config3"] = precision_accuracy(plr, torch, dev)
        if not args.no_batching:
            extra["batching_256"] = batching_run(plr, torch, dev, max(5, args.steps), max(3, args.warmup),
                                                 ck.get("sm_max_mhz"))
        if not args.no_serving:
            extra["serving"] = serving_run(plr, torch, dev, args.serve_jobs, args.serve_sweeps,
                                           int(args.serve_budget_mib * 2 ** 20))
        if not args.no_paper:
            extra["paper_protocol"] = paper_run(plr, torch, dev, seconds_per_case=1.0, Ls=(1024, 4096), scan=False)

    e2e = timed_e2e(plr, torch, specs, max(3, args.steps // 3), 1, dev)
    if world > 1:  # every rank runs the same amount of work: the slowest rank's rate, times the ranks
        e2e["value"] = rank_min(e2e["value"], world, dev) * world

    if rank == 0:
        cpu = cpu_baseline(specs, args.cpu_seconds) if world == 1 else None
        nslots = sum(s.R for s in specs)
        plan = 1 if nslots > torch.cuda.get_device_properties(dev).multi_processor_count else 0
        launches = args.steps * (SWEEPS_PER_STEP * (2 + plan) + 1)  # (plan +) sweep + exchange, then measure
        desc = dict(desc)
        desc["precision"] = prec
        desc["l2"] = "flushed between timed steps (512 MB write)"
        desc["parallelism"] = ("one CTA per temperature slot at a time, persistent CTAs placed on SMs by "
                               "expected work; %d slots per GPU" % nslots)
        line = {"metric": "spin-flip attempts/s", "value": value, "unit": "attempts/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": {"fp64": "f64", "fp32": "f32", "fx64": "int64"}[prec], "data": "synthetic", "config": desc,
                "clocks": ck, "e2e": e2e, "gpu_launches": launches, "roofline": roof,
                "cpu_baseline": cpu, "acceptance": A}
        line.update(extra)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
