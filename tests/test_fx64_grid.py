"""The fixed-point grid of the FX64 precision mode, checked on the CPU with exact
integer arithmetic against the oracle's FP64 couplings (no GPU).

The mode keeps local fields as 64-bit integers in units of 2^-F, F = 61 - e
with Jtot < 2^e, built from the couplings rounded to the grid, Jx(r) =
round(J*(r) 2^F).  Its claims, pinned here for shapes across the supported
range:
  * no field, field difference or corrected difference leaves int64: every
    field is at most sum_r Jx(r) < 2^62;
  * an energy difference computed from the integer fields is within
    L 2^-(F+1) <= L 2^-61 Jtot of the same difference in exact arithmetic on
    the FP64 couplings, far inside the 1e-9 near-tie band of the acceptance
    rule (Eq. 8) for every temperature of the workloads.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle


def _grid(jtot):
    m, e = math.frexp(jtot)  # jtot = m 2^e, m in [0.5, 1)
    return 61 - max(e, 0)


def _rounded(J, F):
    return [int(round(Fraction(float(v)) * 2 ** F)) for v in J]


@pytest.mark.parametrize("L,sigma", [(2, 0.5), (64, 0.5), (1024, 0.4), (4096, 0.2), (16384, 0.1), (65536, 0.1),
                                     (65536, 1.0), (1000, 0.02), (300, 3.0)])
def test_fx64_fields_fit_int64(L, sigma):
    J = oracle.jstar(L, sigma)
    jtot = float(np.sum(J[1:]))
    F = _grid(jtot)
    assert F >= 24
    Jx = _rounded(J, F)
    assert Jx[0] == 0
    top = sum(Jx[1:])  # the largest field: every other site in the same state
    assert top < 2 ** 62
    # each rounded coupling is within half a unit of the FP64 one (exact check)
    for r in (1, 2, L // 3, L // 2, L - 1):
        if 0 < r < L:
            assert abs(Fraction(Jx[r]) - Fraction(float(J[r])) * 2 ** F) <= Fraction(1, 2)


@pytest.mark.parametrize("L,q,sigma,seed", [(64, 3, 0.5, 1), (257, 4, 0.15, 2), (1024, 5, 0.4, 3),
                                            (2048, 8, 0.1, 4)])
def test_fx64_energy_difference_bound(L, q, sigma, seed):
    """For random configurations and proposals, the exact integer difference
    d_fx = h[a][k] - h[b][k] (in units of 2^-F) agrees with the exact rational
    value of the same difference on the FP64 couplings within L 2^-(F+1)."""
    J = oracle.jstar(L, sigma)
    jtot = float(np.sum(J[1:]))
    F = _grid(jtot)
    Jx = _rounded(J, F)
    rng = np.random.default_rng(seed)
    s = rng.integers(0, q, size=L)
    bound = Fraction(L, 2 ** (F + 1))
    assert bound <= Fraction(L) * Fraction(jtot) / 2 ** 61
    Jf = [Fraction(float(v)) for v in J]
    for k in rng.integers(0, L, size=12):
        a = int(s[k])
        b = (a + 1 + int(rng.integers(0, q - 1))) % q
        dx = 0
        de = Fraction(0)
        for j in range(L):
            r = (k - j) % L
            c = int(s[j] == a) - int(s[j] == b)
            if c:
                dx += c * Jx[r]
                de += c * Jf[r]
        err = abs(Fraction(dx, 2 ** F) - de)
        assert err <= bound
    # the bound is below 1e-9 / (beta c) for the coldest temperature of the
    # workloads (T = 0.02 Jtot, c = 2): the decisions can differ from FP64
    # mode's only inside the counted near-tie band
    assert float(bound) * 2 / (0.02 * jtot) < 1e-9
