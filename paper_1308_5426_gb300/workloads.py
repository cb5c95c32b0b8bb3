"""Seeded synthetic inputs for the long-range Potts PT workloads.

This module holds only input recipes (sizes, temperature ratios, seeds, job
draws, arrival traces).  It performs none of the method's arithmetic: absolute
temperatures are T_t = ratio_t * Jtot, and each side (the GPU library and the
CPU oracle) forms Jtot from its own J* table.  Both the tests and the benchmark
draw their inputs from here.

The paper's runs (Sec. 5) use q = 3, L = 512..10240, 400 replicas and a uniform
temperature grid; the workloads below keep those shapes where they are named
and use geometric grids in units of Jtot = sum_r J*(r) otherwise.
"""
from dataclasses import dataclass

import numpy as np


def geometric_ratios(R: int, lo: float, hi: float) -> np.ndarray:
    """T_t / Jtot = lo * (hi/lo)^(t/(R-1)), t = 0..R-1, ascending."""
    if R == 1:
        return np.array([lo], dtype=np.float64)
    t = np.arange(R, dtype=np.float64)
    return lo * (hi / lo) ** (t / (R - 1))


def uniform_ratios(R: int, lo: float, hi: float) -> np.ndarray:
    """Uniform grid (the paper's choice in Sec. 5.1), ascending."""
    return np.linspace(lo, hi, R, dtype=np.float64)


@dataclass
class JobSpec:
    L: int
    q: int
    sigma: float
    ratios: np.ndarray          # T/Jtot per slot, ascending
    seed: int
    sweeps: int
    measure_every: int = 10
    c: int = 2
    precision: str = "fp64"    # "fp64" or "fp32"
    arrival: float = 0.0        # seconds since trace start (serving only)

    @property
    def R(self) -> int:
        return int(self.ratios.size)

    @property
    def attempts(self) -> int:
        return self.L * self.R * self.sweeps

    @property
    def field_bytes(self) -> int:
        """Admission footprint of the serving workload: L * q * R * 4 bytes."""
        return self.L * self.q * self.R * 4


def parity_job(sweeps: int = 1000) -> JobSpec:
    """Small plain-FP64 PT job: L=64, q=3, sigma=0.5, R=16, T/Jtot in [0.05, 1]."""
    return JobSpec(L=64, q=3, sigma=0.5, ratios=geometric_ratios(16, 0.05, 1.0), seed=1,
                   sweeps=sweeps)


def chains_jobs(sweeps: int = 10_000) -> list:
    """Eight independent plain-FP64 chains: L=1024, q=5, sigma=0.4, R=64, seeds 1..8,
    measured every 10 sweeps."""
    return [JobSpec(L=1024, q=5, sigma=0.4, ratios=geometric_ratios(64, 0.05, 1.0), seed=s,
                    sweeps=sweeps, measure_every=10) for s in range(1, 9)]


def precision_job(precision: str = "fp32", sweeps: int = 10_000) -> JobSpec:
    """Mixed-precision job: L=4096, q=8, sigma=0.2, R=128, T/Jtot in [0.02, 0.5]."""
    return JobSpec(L=4096, q=8, sigma=0.2, ratios=geometric_ratios(128, 0.02, 0.5), seed=1,
                   sweeps=sweeps, precision=precision)


def batching_jobs(n: int = 256, seed: int = 4, sweeps: int = 2000) -> list:
    """Ragged batch: L uniform in {256, 512, ..., 8192}, q uniform in 2..10,
    sigma uniform in [0.1, 1.0], R uniform in {32, 64, 128}, T/Jtot in [0.05, 1],
    FP32 fields; job j has seed j+1."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Ls = 256 * rng.integers(1, 33, size=n)
    qs = rng.integers(2, 11, size=n)
    sig = rng.uniform(0.1, 1.0, size=n)
    Rs = rng.choice(np.array([32, 64, 128]), size=n)
    return [JobSpec(L=int(Ls[j]), q=int(qs[j]), sigma=float(sig[j]),
                    ratios=geometric_ratios(int(Rs[j]), 0.05, 1.0), seed=j + 1, sweeps=sweeps,
                    precision="fp32") for j in range(n)]


def serving_trace(n: int = 500, rate: float = 50.0, seed: int = 5, sweeps: int = 5000) -> list:
    """Poisson arrivals at `rate` jobs/s of phase-diagram points: q in {3, 5, 8},
    sigma uniform in [0.1, 1.0], L in {512, ..., 16384} (powers of two), R = 64,
    T/Jtot in [0.05, 1], FP32 fields; job j has seed j+1."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate, size=n)
    arrivals = np.cumsum(gaps) - gaps[0]
    qs = rng.choice(np.array([3, 5, 8]), size=n)
    sig = rng.uniform(0.1, 1.0, size=n)
    Ls = 2 ** rng.integers(9, 15, size=n)
    return [JobSpec(L=int(Ls[j]), q=int(qs[j]), sigma=float(sig[j]),
                    ratios=geometric_ratios(64, 0.05, 1.0), seed=j + 1, sweeps=sweeps,
                    precision="fp32", arrival=float(arrivals[j])) for j in range(n)]


def paper_benchmark_jobs() -> list:
    """The paper's benchmark shapes (Sec. 5.2): q = 3, L = 512..10240, 400 replicas,
    10^4 production sweeps at L = 512 down to 50 at L = 10240 (plus 20 %
    thermalisation), sigma = 0.2, uniform temperature grid."""
    Ls = [512, 1024, 2048, 3072, 4096, 5120, 6144, 8192, 10240]
    out = []
    for L in Ls:
        prod = max(50, int(round(1e4 * (512.0 / L) ** 2)))
        out.append(JobSpec(L=L, q=3, sigma=0.2, ratios=uniform_ratios(400, 0.1, 1.0), seed=1,
                           sweeps=int(prod * 1.2), precision="fp32"))
    return out
