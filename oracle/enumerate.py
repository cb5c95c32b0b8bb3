"""Exact Boltzmann averages by enumeration of all q^L configurations.

TEST INFRASTRUCTURE (see oracle/__init__.py).  Written straight from the
definitions: H of Eq. 2 (with pair factor c), the Boltzmann weight
exp(-beta H) of the canonical ensemble the Metropolis rule of Eq. 8 samples,
and M of Eq. 10.  Usable for q^L up to a few 10^4 states.
"""
import itertools

import numpy as np


def all_states(L: int, q: int) -> np.ndarray:
    return np.array(list(itertools.product(range(q), repeat=L)), dtype=np.int64)


def energies(states: np.ndarray, J: np.ndarray, c: int) -> np.ndarray:
    """E = -(c/2) sum_{i != j} J*(|i-j|) delta(s_i, s_j) for each row (Eq. 2)."""
    L = states.shape[1]
    idx = np.arange(L)
    Jmat = J[np.abs(idx[:, None] - idx[None, :])]  # J[0] = 0 on the diagonal
    eq = states[:, :, None] == states[:, None, :]
    return -0.5 * c * np.einsum("nij,ij->n", eq.astype(np.float64), Jmat)


def magnetisations(states: np.ndarray, q: int) -> np.ndarray:
    """M = (q N_max / L - 1) / (q - 1) for each row (Eq. 10)."""
    L = states.shape[1]
    counts = np.stack([(states == x).sum(axis=1) for x in range(q)], axis=1)
    return (q * counts.max(axis=1) / L - 1.0) / (q - 1.0)


def exact_averages(L: int, q: int, J: np.ndarray, c: int, betas) -> dict:
    """<E>, <E^2>, <E^4>, <M>, <M^2>, <M^4> at each beta, exactly."""
    S = all_states(L, q)
    E = energies(S, J, c)
    M = magnetisations(S, q)
    out = {k: [] for k in ("E", "E2", "E4", "M", "M2", "M4")}
    for beta in betas:
        w = np.exp(-beta * (E - E.min()))  # shift for range; cancels in ratios
        Z = w.sum()
        out["E"].append((w * E).sum() / Z)
        out["E2"].append((w * E * E).sum() / Z)
        out["E4"].append((w * E ** 4).sum() / Z)
        out["M"].append((w * M).sum() / Z)
        out["M2"].append((w * M ** 2).sum() / Z)
        out["M4"].append((w * M ** 4).sum() / Z)
    return {k: np.array(v) for k, v in out.items()}
