"""Periodic long-range couplings J*(r) for the oracle, written from Eq. 6.

TEST INFRASTRUCTURE (see oracle/__init__.py).

    J*(r) = r^{-s} + L^{-s} [ zeta(s, 1 + r/L) + zeta(s, 1 - r/L) ],  s = 1 + sigma,

with zeta(s, a) the Hurwitz zeta function of Eq. 7, evaluated here by the
library routine scipy.special.zeta (a library primitive used as one step).
J*(0) is set to 0: the Hamiltonian of Eq. 2 excludes i = j.
"""
import numpy as np
from scipy.special import zeta


def jstar(L: int, sigma: float) -> np.ndarray:
    """Return J*(r) for r = 0..L-1 as float64, J*(0) = 0 (Eq. 6)."""
    if L < 2 or not sigma > 0:
        raise ValueError("need L >= 2 and sigma > 0")
    s = 1.0 + float(sigma)
    r = np.arange(1, L, dtype=np.float64)
    out = np.zeros(L, dtype=np.float64)
    out[1:] = r ** (-s) + float(L) ** (-s) * (zeta(s, 1.0 + r / L) + zeta(s, 1.0 - r / L))
    return out


def jtot(L: int, sigma: float) -> float:
    """Jtot = sum_{r=1}^{L-1} J*(r), the field scale sum_x h[x][i]."""
    return float(np.sum(jstar(L, sigma)[1:]))
