"""Plain CPU FP64 oracle for long-range Potts parallel tempering (arXiv:1308.5426).

TEST INFRASTRUCTURE.  This package is the slow, obviously-correct reference the
GPU library is checked against.  Only the test suite, the package-entry smoke
check and the CPU-baseline leg of the benchmark may import it; the product
path never does.  It shares no code with the GPU library:

  * oracle/potts_oracle.c -- the Markov chain itself (Eq. 2, 8, 9, 10, Sec. 4.2),
    its own Philox4x32-10, energies by the plain double sum;
  * oracle/jstar.py       -- J*(r) from Eq. 6 with scipy's Hurwitz zeta;
  * oracle/enumerate.py   -- exact Boltzmann averages by enumeration.

Pins (tests marked "not gpu"): J* against the image sum of Eq. 5 with its
integral tail, against mpmath and against closed forms; Philox against curand's
host generator; energies against the ordered ground state, the infinite-
temperature mean and a worked example; the dynamics against exact enumeration.
"""
import ctypes

import numpy as np

from . import build as _build
from .jstar import jstar, jtot  # noqa: F401

_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(_build.build())
    P = ctypes.c_void_p
    lib.oracle_create.restype = P
    lib.oracle_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P, ctypes.c_int, P,
                                  ctypes.c_uint64, ctypes.c_int]
    lib.oracle_destroy.argtypes = [P]
    lib.oracle_sweep.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.oracle_sweep.restype = ctypes.c_int
    lib.oracle_exchange.argtypes = [P]
    lib.oracle_energy_direct.argtypes = [P, ctypes.c_int]
    lib.oracle_energy_direct.restype = ctypes.c_double
    lib.oracle_magnetisation.argtypes = [P, ctypes.c_int]
    lib.oracle_magnetisation.restype = ctypes.c_double
    lib.oracle_get_spins.argtypes = [P, P]
    lib.oracle_set_spins.argtypes = [P, P]
    lib.oracle_get_running_energy.argtypes = [P, P]
    lib.oracle_get_fields.argtypes = [P, P]
    lib.oracle_set_counters.argtypes = [P, ctypes.c_uint32, ctypes.c_uint32]
    lib.oracle_set_random_sites.argtypes = [P, ctypes.c_int]
    lib.oracle_get_counters.argtypes = [P, P, P]
    lib.oracle_get_stats.argtypes = [P] * 8
    lib.oracle_philox.argtypes = [P, P, P]
    lib.oracle_set_overrides.argtypes = [P, P, ctypes.c_int]
    lib.oracle_set_overrides.restype = ctypes.c_int
    lib.oracle_get_near_log.argtypes = [P, P, ctypes.c_int]
    lib.oracle_get_near_log.restype = ctypes.c_uint64
    lib.oracle_get_adopted.argtypes = [P] * 5
    _lib = lib
    return lib


def philox4x32_10(ctr, key):
    """Raw Philox4x32-10 block of the oracle's own generator (for its pin)."""
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.oracle_philox(c.ctypes.data, k.ctypes.data, out.ctypes.data)
    return out


class Oracle:
    """One parallel-tempering job: R temperature slots of an L-site, q-state chain.

    temps: absolute temperatures (k_B = 1), ascending, slot t gets beta_t = 1/T_t.
    c: pair factor of Eq. 2 (2 = ordered i != j double sum, 1 = each pair once).
    fields: keep incremental local fields (needed for mode="field").
    J: optional J* table (defaults to oracle.jstar(L, sigma)).
    site_order: "sequential" (sites 0..L-1 in order) or "random" (attempt m of
    a sweep at site floor(x3 L / 2^32) of Philox counter (m, t, n, 3)).
    """

    def __init__(self, L, q, sigma, temps, seed, c=2, fields=True, J=None, site_order="sequential"):
        lib = _load()
        self.L, self.q, self.c = int(L), int(q), int(c)
        self.sigma = float(sigma)
        self.temps = np.ascontiguousarray(temps, dtype=np.float64)
        self.R = int(self.temps.size)
        if np.any(~np.isfinite(self.temps)) or np.any(self.temps <= 0):
            raise ValueError("temperatures must be positive and finite")
        self.beta = np.ascontiguousarray(1.0 / self.temps)
        self.J = np.ascontiguousarray(jstar(self.L, self.sigma) if J is None else J, dtype=np.float64)
        self.seed = int(seed)
        self._fields = bool(fields)
        self._h = lib.oracle_create(self.L, self.q, self.c, self.J.ctypes.data, self.R,
                                    self.beta.ctypes.data, ctypes.c_uint64(self.seed),
                                    int(self._fields))
        if not self._h:
            raise ValueError("oracle_create rejected its arguments")
        if site_order not in ("sequential", "random"):
            raise ValueError("site_order must be 'sequential' or 'random'")
        lib.oracle_set_random_sites(self._h, int(site_order == "random"))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.oracle_destroy(h)
            self._h = None

    def sweep(self, n=1, mode="field", nthreads=1):
        m = {"direct": 0, "field": 1}[mode]
        rc = _lib.oracle_sweep(self._h, int(n), m, int(nthreads))
        if rc != 0:
            raise RuntimeError("oracle_sweep failed (%d)" % rc)

    def exchange(self):
        _lib.oracle_exchange(self._h)

    def step(self, mode="field", nthreads=1):
        """One sweep of every slot followed by one exchange step."""
        self.sweep(1, mode, nthreads)
        self.exchange()

    def spins(self):
        out = np.zeros((self.R, self.L), dtype=np.uint8)
        _lib.oracle_get_spins(self._h, out.ctypes.data)
        return out

    def set_spins(self, s):
        s = np.ascontiguousarray(s, dtype=np.uint8).reshape(self.R, self.L)
        _lib.oracle_set_spins(self._h, s.ctypes.data)

    def running_energy(self):
        out = np.zeros(self.R, dtype=np.float64)
        _lib.oracle_get_running_energy(self._h, out.ctypes.data)
        return out

    def energy(self):
        """Energies of every slot by the plain O(L^2) double sum (Eq. 2)."""
        return np.array([_lib.oracle_energy_direct(self._h, t) for t in range(self.R)])

    def magnetisation(self):
        return np.array([_lib.oracle_magnetisation(self._h, t) for t in range(self.R)])

    def fields(self):
        if not self._fields:
            raise RuntimeError("oracle created without fields")
        out = np.zeros((self.R, self.q, self.L), dtype=np.float64)
        _lib.oracle_get_fields(self._h, out.ctypes.data)
        return out

    def counters(self):
        ns = ctypes.c_uint32()
        ne = ctypes.c_uint32()
        _lib.oracle_get_counters(self._h, ctypes.byref(ns), ctypes.byref(ne))
        return ns.value, ne.value

    def set_counters(self, nsweep, nexch):
        _lib.oracle_set_counters(self._h, int(nsweep), int(nexch))

    def set_overrides(self, events):
        """Decisions to adopt where the oracle itself sees a near tie (the
        re-synchronisation of two FP64 implementations whose exp and log round
        differently): rows {kind (0 Metropolis, 1 exchange), slot t (exchange:
        pair (t, t+1)), sweep n (exchange: index m), attempt within the sweep
        (exchange: stage), decision (0/1)}.  Replaces the previous table."""
        ev = np.ascontiguousarray(np.asarray(events, dtype=np.int32).reshape(-1, 5))
        if _lib.oracle_set_overrides(self._h, ev.ctypes.data if ev.size else None, int(ev.shape[0])) != 0:
            raise MemoryError("oracle_set_overrides")

    def near_log(self):
        """Near-tie events seen so far, rows {kind, slot or pair, sweep or
        exchange index, attempt or stage, own decision, decision taken}, and
        the total count (the log keeps the first 4096)."""
        cap = 4096
        out = np.zeros((cap, 6), np.int32)
        n = int(_lib.oracle_get_near_log(self._h, out.ctypes.data, cap))
        return out[: min(n, cap)].copy(), n

    def adopted(self):
        """Adopted near-tie decisions: per slot (Metropolis) and for the
        exchange, all of them and those that reversed the oracle's own."""
        am = np.zeros(self.R, np.uint64)
        fm = np.zeros(self.R, np.uint64)
        ae = np.zeros(1, np.uint64)
        fe = np.zeros(1, np.uint64)
        _lib.oracle_get_adopted(self._h, am.ctypes.data, fm.ctypes.data, ae.ctypes.data, fe.ctypes.data)
        return {"metro": am, "metro_reversed": fm, "exch": int(ae[0]), "exch_reversed": int(fe[0])}

    def stats(self):
        R = self.R
        acc = np.zeros(R, np.uint64)
        att_sw = np.zeros(R, np.uint64)
        acc_sw = np.zeros(R, np.uint64)
        near = np.zeros(R, np.uint64)
        first = np.zeros(R, np.int64)
        ne = np.zeros(1, np.uint64)
        fe = np.zeros(1, np.int64)
        _lib.oracle_get_stats(self._h, acc.ctypes.data, att_sw.ctypes.data, acc_sw.ctypes.data,
                              near.ctypes.data, first.ctypes.data, ne.ctypes.data, fe.ctypes.data)
        return {"acc_flip": acc, "att_swap": att_sw[: max(R - 1, 0)], "acc_swap": acc_sw[: max(R - 1, 0)],
                "near_metro": near, "first_near_metro": first,
                "near_exch": int(ne[0]), "first_near_exch": int(fe[0])}
