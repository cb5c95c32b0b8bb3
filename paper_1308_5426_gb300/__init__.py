"""GB300-native parallel-tempering Metropolis simulation of the 1D long-range
q-state Potts chain (A. Boer, arXiv:1308.5426), on one GPU.

The compute path lives in the CUDA library libpotts_lr.so (C ABI in
include/potts_lr.h); this module only marshals arguments to it.

    import paper_1308_5426_gb300 as plr
    job = plr.Job(L=1024, q=5, sigma=0.4, temps=T, seed=1)   # FP64 reference mode
    for n in range(steps):
        job.sweep(1); job.exchange()
    E, M = job.measure()
"""
import ctypes

import numpy as np

from . import _lib
from ._lib import FP32, FP64, FX64, PottsError  # noqa: F401

__all__ = ["Job", "Batch", "jstar", "jtot", "FP32", "FP64", "FX64", "PottsError"]


def jstar(L: int, sigma: float) -> np.ndarray:
    """J*(r), r = 0..L-1 (Eq. 6), from the library's FP64 Euler-Maclaurin builder."""
    lib = _lib.load()
    out = np.zeros(int(L), dtype=np.float64)
    _lib.check(lib.potts_lr_jstar(int(L), float(sigma), _lib._ptr(out)))
    return out


def jtot(L: int, sigma: float) -> float:
    return float(jstar(L, sigma)[1:].sum())


def probe(what: str) -> float:
    """Measured throughput of this GPU: "fp64_add", "fp32_add", "i64_add"
    (adds/s), "smem" or "l2" (bytes/s loaded + stored) -- roofline
    denominators."""
    lib = _lib.load()
    v = ctypes.c_double()
    _lib.check(lib.potts_lr_probe({"fp64_add": 0, "fp32_add": 1, "smem": 2, "l2": 3, "i64_add": 4}[what],
                                  ctypes.byref(v)))
    return v.value


SWEEP_VARIANTS = ("auto", "memory", "registers", "global", "direct", "cluster", "rcluster") + tuple(
    "registers%d" % c for c in range(1, 9))


def sweep_variant_code(name):
    """potts_lr_opts.sweep_variant for a variant name: "auto", "memory",
    "registers", "global", "direct" (the paper's O(L)-per-attempt sweep, FP64),
    "cluster" (a slot's fields shared by a cluster of 2, 4 or 8 CTAs in shared
    memory), "rcluster" (the same in the CTAs' registers; FP32 and FX64) or
    "registers<c>" (register configuration c = 1..8)."""
    if name in ("auto", "memory", "registers", "global", "direct", "cluster", "rcluster"):
        return {"auto": 0, "memory": 1, "registers": 2, "global": 3, "direct": 4, "cluster": 5, "rcluster": 6}[name]
    if isinstance(name, str) and name.startswith("registers") and name[9:].isdigit() and 1 <= int(name[9:]) <= 8:
        return 16 + int(name[9:])
    raise ValueError("unknown sweep variant %r" % (name,))


class Job:
    """One PT job on the GPU (potts_lr_create).

    temps: absolute temperatures, ascending (slot order); precision "fp64",
    "fp32" or "fx64" (64-bit fixed-point fields: exact integer updates, FP64
    decisions, no drift); recompute_every: FP32 tensor-core field rebuild interval K;
    pair_factor: c of Eq. 2; stream: optional cudaStream_t handle as an int
    (e.g. torch.cuda.current_stream().cuda_stream); sweep_variant: "auto",
    "memory" or "registers" (FP32 field residency), "global" (fields in global
    memory even where they fit in shared memory), "registers<c>" (register
    configuration c) -- all give identical results (see tune.py for a tuner);
    site_order: "sequential" or "random" (attempts at Philox-drawn sites; FP64,
    direct sweep).
    """

    def __init__(self, L, q, sigma, temps, seed, precision="fp64", recompute_every=100, pair_factor=2,
                 stream=None, sweep_variant="auto", site_order="sequential"):
        lib = _lib.load()
        self.L, self.q, self.sigma = int(L), int(q), float(sigma)
        self.temps = np.ascontiguousarray(temps, dtype=np.float64)
        self.R = int(self.temps.size)
        self.seed = int(seed)
        self.precision = precision
        o = _lib.Opts()
        lib.potts_lr_default_opts(ctypes.byref(o))
        o.precision = _lib.PRECISIONS[precision]
        o.recompute_every = int(recompute_every)
        o.pair_factor = int(pair_factor)
        o.cuda_stream = ctypes.c_void_p(int(stream)) if stream else None
        o.sweep_variant = sweep_variant_code(sweep_variant)
        o.site_order = {"sequential": 0, "random": 1}[site_order]
        h = ctypes.c_void_p()
        _lib.check(lib.potts_lr_create(self.L, self.q, self.sigma, _lib._ptr(self.temps), self.R,
                                       ctypes.c_uint64(self.seed), ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        self._lib = lib

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.potts_lr_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sweep(self, n=1):
        _lib.check(self._lib.potts_lr_sweep(self._h, int(n)))

    def exchange(self):
        _lib.check(self._lib.potts_lr_exchange(self._h))

    def measure(self, E=None, M=None):
        """Energies and magnetisations per slot (host arrays, optionally caller-owned)."""
        E = np.zeros(self.R) if E is None else E
        M = np.zeros(self.R) if M is None else M
        _lib.check(self._lib.potts_lr_measure(self._h, _lib._ptr(E), _lib._ptr(M)))
        return E, M

    def measure_device(self, E_ptr, M_ptr):
        _lib.check(self._lib.potts_lr_measure_device(self._h, ctypes.c_void_p(E_ptr), ctypes.c_void_p(M_ptr)))

    def fields_recompute(self):
        _lib.check(self._lib.potts_lr_fields_recompute(self._h))

    def fields_error(self):
        v = ctypes.c_double()
        _lib.check(self._lib.potts_lr_fields_error(self._h, ctypes.byref(v)))
        return v.value

    def get_state(self) -> bytes:
        n = ctypes.c_size_t()
        _lib.check(self._lib.potts_lr_get_state(self._h, None, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        _lib.check(self._lib.potts_lr_get_state(self._h, buf, ctypes.byref(n)))
        return buf.raw[: n.value]

    def set_state(self, state: bytes):
        _lib.check(self._lib.potts_lr_set_state(self._h, state, len(state)))

    def state_size(self) -> int:
        n = ctypes.c_size_t()
        _lib.check(self._lib.potts_lr_get_state(self._h, None, ctypes.byref(n)))
        return n.value

    def get_state_into(self, ptr: int, nbytes: int):
        """Checkpoint into caller memory at host address ptr (e.g. pinned)."""
        n = ctypes.c_size_t(nbytes)
        _lib.check(self._lib.potts_lr_get_state(self._h, ctypes.c_void_p(ptr), ctypes.byref(n)))

    def set_state_from(self, ptr: int, nbytes: int):
        _lib.check(self._lib.potts_lr_set_state(self._h, ctypes.c_void_p(ptr), int(nbytes)))

    def spins(self):
        out = np.zeros((self.R, self.L), dtype=np.uint8)
        _lib.check(self._lib.potts_lr_get_spins(self._h, _lib._ptr(out)))
        return out

    def fields(self):
        out = np.zeros((self.R, self.q, self.L), dtype=np.float64)
        _lib.check(self._lib.potts_lr_get_fields(self._h, _lib._ptr(out)))
        return out

    def running_energy(self):
        out = np.zeros(self.R)
        _lib.check(self._lib.potts_lr_get_energy(self._h, _lib._ptr(out)))
        return out

    def stats(self):
        acc = np.zeros(self.R, np.uint64)
        sw = np.zeros(self.R, np.uint64)
        near = np.zeros(2, np.uint64)
        _lib.check(self._lib.potts_lr_stats(self._h, _lib._ptr(acc), _lib._ptr(sw), _lib._ptr(near)))
        return {"acc_flip": acc, "acc_swap": sw[: max(self.R - 1, 0)], "near_metro": int(near[0]),
                "near_exch": int(near[1])}

    def sweep_info(self):
        """The sweep kernel this job runs (potts_lr_sweep_info)."""
        v = np.zeros(7, np.int32)
        _lib.check(self._lib.potts_lr_sweep_info(self._h, _lib._ptr(v), 7))
        kind = ("memory", "registers", "cluster", "direct", "register_cluster")[int(v[0])]
        return {"kernel": kind, "fields_in_smem": bool(v[1]), "table_in_smem": bool(v[2]),
                "register_config": int(v[3]), "cluster": int(v[4]), "threads": int(v[5]),
                "smem_bytes": int(v[6])}

    def set_rebuild_split(self, parts):
        """FP32: BF16 parts of J* in the tensor-core rebuild: 3, 2, or 0 (default:
        2 while scheduled rebuilds come every sweep, else 3)."""
        _lib.check(self._lib.potts_lr_set_rebuild_split(self._h, int(parts)))

    def rebuild_info(self):
        """FP32 rebuild schedule: current interval (sweeps), automatic rebuilds
        done, drift of the last one (/ Jtot)."""
        k, n, d = ctypes.c_int32(), ctypes.c_uint32(), ctypes.c_double()
        _lib.check(self._lib.potts_lr_rebuild_info(self._h, ctypes.byref(k), ctypes.byref(n), ctypes.byref(d)))
        return {"interval": k.value, "rebuilds": n.value, "last_drift": d.value}

    def set_wait_limits(self, rebuild_ns=4_000_000_000, plan_ns=50_000):
        """Bounds of the device waits (potts_lr_set_wait_limits); small values
        make them expire (the tests of the failure paths)."""
        _lib.check(self._lib.potts_lr_set_wait_limits(self._h, ctypes.c_uint64(int(rebuild_ns)),
                                                      ctypes.c_uint64(int(plan_ns))))

    def near_log(self):
        """Near ties so far (potts_lr_near_log): rows {kind (0 Metropolis, 1
        exchange), slot or pair, sweep or exchange index, attempt or stage,
        decision}, and the number logged since create."""
        out = np.zeros((_lib.NEAR_LOG_CAP, 5), np.int32)
        n = ctypes.c_int()
        _lib.check(self._lib.potts_lr_near_log(self._h, _lib._ptr(out), _lib.NEAR_LOG_CAP, ctypes.byref(n)))
        return out[: min(n.value, _lib.NEAR_LOG_CAP)].copy(), n.value

    def counters(self):
        a, b = ctypes.c_uint32(), ctypes.c_uint32()
        _lib.check(self._lib.potts_lr_counters(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def sync(self):
        _lib.check(self._lib.potts_lr_sync(self._h))


class Batch:
    """Many jobs stepped together (potts_lr_batch_*): one step = one sweep of
    every slot of every job + one exchange step per job, graph-captured."""

    def __init__(self, jobs, stream=None):
        lib = _lib.load()
        self.jobs = list(jobs)
        arr = (ctypes.c_void_p * len(self.jobs))(*[j.handle.value for j in self.jobs])
        h = ctypes.c_void_p()
        st = ctypes.c_void_p(int(stream)) if stream else None
        _lib.check(lib.potts_lr_batch_create(arr, len(self.jobs), st, ctypes.byref(h)))
        self._h = h
        self._lib = lib

    @property
    def nslots(self):
        return sum(j.R for j in self.jobs)

    def run(self, nsteps, steps_per_graph=10):
        _lib.check(self._lib.potts_lr_batch_run(self._h, int(nsteps), int(steps_per_graph)))

    def sweep(self, n=1):
        _lib.check(self._lib.potts_lr_batch_sweep(self._h, int(n)))

    def exchange(self):
        _lib.check(self._lib.potts_lr_batch_exchange(self._h))

    def measure(self):
        """Energies and magnetisations of every slot, job order then slot order."""
        E = np.zeros(self.nslots)
        M = np.zeros(self.nslots)
        _lib.check(self._lib.potts_lr_batch_measure(self._h, _lib._ptr(E), _lib._ptr(M)))
        return E, M

    def measure_device(self, E_ptr, M_ptr):
        _lib.check(self._lib.potts_lr_batch_measure_device(self._h, ctypes.c_void_p(E_ptr),
                                                            ctypes.c_void_p(M_ptr)))

    def sync(self):
        _lib.check(self._lib.potts_lr_batch_sync(self._h))

    def state_size(self) -> int:
        """Bytes of the batch checkpoint (the jobs' checkpoints back to back)."""
        n = ctypes.c_size_t()
        _lib.check(self._lib.potts_lr_batch_state_size(self._h, ctypes.byref(n)))
        return n.value

    def get_state_into(self, ptr: int, nbytes: int):
        """Checkpoint every job into caller memory at host address ptr (e.g.
        pinned), one synchronisation."""
        _lib.check(self._lib.potts_lr_batch_get_state(self._h, ctypes.c_void_p(ptr), int(nbytes)))

    def set_state_from(self, ptr: int, nbytes: int):
        _lib.check(self._lib.potts_lr_batch_set_state(self._h, ctypes.c_void_p(ptr), int(nbytes)))

    def get_state(self) -> bytes:
        n = self.state_size()
        buf = ctypes.create_string_buffer(n)
        self.get_state_into(ctypes.addressof(buf), n)
        return buf.raw[:n]

    def set_state(self, state: bytes):
        buf = ctypes.create_string_buffer(state, len(state))
        self.set_state_from(ctypes.addressof(buf), len(state))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.potts_lr_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
