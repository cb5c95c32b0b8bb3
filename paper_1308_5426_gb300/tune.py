"""Autotuner of the sweep kernel's shape: for a job shape (L, q, precision) it
times the library's automatic choice and every sweep variant that can hold
it -- fields in shared memory, in
global memory, in the shared memory of a cluster of CTAs, in the registers of
a cluster (FP32 and FX64), and each single-CTA register configuration (E sites
per update thread x update warps; FP32 and FX64) --
on this GPU and keeps the fastest.

All variants give bit-identical results, so the choice affects speed only.
Each candidate sweeps a probe job of the same shape (its own seed, the job's
temperature ratios) from random spins: `warm` sweeps + exchanges untimed, then
`sweeps` timed with CUDA events on its stream.  Results are cached per shape
for the process, and in a JSON file if one is given.
"""
import json
import os
import threading

import numpy as np

from . import SWEEP_VARIANTS, Job, PottsError

_lock = threading.Lock()
_cache = {}


def candidates(L, q, precision):
    """Variant names that might hold a job of this shape (the library refuses
    those that do not; the tuner skips them).  "auto" comes first: the
    library's own choice, which can also size a cluster beyond what its fields
    need (a cluster asked for by name keeps the smallest size)."""
    regs = [v for v in SWEEP_VARIANTS if v.startswith("registers") and v != "registers"]
    if precision == "fp64":
        return ["auto", "memory", "global", "cluster"]
    if precision == "fx64":
        return ["auto", "memory", "global", "cluster", "rcluster"] + regs[:6]  # FX64 register configurations 1..6
    return ["auto", "memory", "global", "cluster", "rcluster"] + regs


def _time_variant(L, q, sigma, temps, variant, precision, sweeps, warm, torch):
    st = torch.cuda.Stream()
    try:
        j = Job(L, q, sigma, temps, 1, precision=precision, recompute_every=0, stream=st.cuda_stream,
                sweep_variant=variant)
    except PottsError:
        return None  # the shape does not fit this variant
    try:
        for _ in range(warm):
            j.sweep(1)
            j.exchange()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(sweeps):
            j.sweep(1)
            j.exchange()
        e1.record(st)
        e1.synchronize()
        return e0.elapsed_time(e1) / sweeps
    finally:
        j.close()


def tune(L, q, sigma=0.5, precision="fp32", R=64, ratios=None, sweeps=4, warm=3, cache_file=None):
    """(best variant name, {variant: ms per sweep}) for this shape.  R and the
    temperature ratios (T/Jtot, default geometric 0.05..1) set the probe job."""
    import torch
    from . import jtot

    key = "%d/%d/%s" % (L, q, precision)
    with _lock:
        if key in _cache:
            return _cache[key]
        if cache_file and os.path.exists(cache_file):
            with open(cache_file) as f:
                disk = json.load(f)
            if key in disk:
                _cache[key] = (disk[key]["best"], disk[key]["ms"])
                return _cache[key]
    if ratios is None:
        ratios = 0.05 * (1.0 / 0.05) ** (np.arange(R) / max(R - 1, 1))
    temps = np.asarray(ratios, dtype=np.float64) * jtot(L, sigma)
    ms = {}
    for v in candidates(L, q, precision):
        t = _time_variant(L, q, sigma, temps, v, precision, sweeps, warm, torch)
        if t is not None:
            ms[v] = t
    best = min(ms, key=ms.get)
    with _lock:
        _cache[key] = (best, ms)
        if cache_file:
            disk = {}
            if os.path.exists(cache_file):
                with open(cache_file) as f:
                    disk = json.load(f)
            disk[key] = {"best": best, "ms": ms}
            with open(cache_file, "w") as f:
                json.dump(disk, f, indent=1, sort_keys=True)
    return best, ms


def best_variant(L, q, precision="fp32", sigma=0.5, cache_file=None):
    """The tuned variant name for a shape (tuning it on first use)."""
    return tune(L, q, sigma=sigma, precision=precision, cache_file=cache_file)[0]
