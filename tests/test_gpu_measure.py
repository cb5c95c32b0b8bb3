"""The energy and magnetisation pass (Eq. 2, Eq. 10) at sizes where one
slot's pair sum is cut into many (r, site) tiles over CTAs, against the
oracle's plain O(L^2) double sum and state counts of the same spins: every
plane count (q = 2, 3..4, 5..8, 9..16), L a multiple of 32 and ragged, both
pair factors."""
import numpy as np
import pytest

import oracle
from paper_1308_5426_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def plr():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1308_5426_gb300
    return paper_1308_5426_gb300


@pytest.mark.parametrize("L,q,c,sweeps", [
    (20001, 12, 2, 0),  # four planes, ragged L: 30 tiles per slot
    (16384, 5, 2, 1),   # three planes, whole 32-site words: 32 tiles
    (12000, 2, 1, 1),   # one plane, pair factor 1
    (9999, 4, 2, 0),    # two planes, ragged
])
def test_tiled_measurement_matches_oracle(plr, L, q, c, sweeps):
    R, sigma = 2, 0.5
    temps = workloads.geometric_ratios(R, 0.05, 1.0) * oracle.jtot(L, sigma)
    j = plr.Job(L, q, sigma, temps, 7, precision="fp32", recompute_every=0, pair_factor=c)
    for _ in range(sweeps):
        j.sweep(1)
        j.exchange()
    E, M = j.measure()
    o = oracle.Oracle(L, q, sigma, temps, 7, c=c, fields=False)
    o.set_spins(j.spins())
    np.testing.assert_allclose(E, o.energy(), rtol=1e-10, atol=0)
    np.testing.assert_allclose(M, o.magnetisation(), rtol=0, atol=1e-14)
    j.close()
