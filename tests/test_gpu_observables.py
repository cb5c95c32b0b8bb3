"""The observables of Sec. 5.1 from GPU chains: U_E (Eq. 11) and V_M (Eq. 12)
per slot, computed by the library's analysis module from the GPU's measured
series, agree with exact enumeration within 3 jackknife errors, in FP64 and in
FP32 mode."""
import numpy as np
import pytest

import oracle
from oracle.enumerate import exact_averages

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def plr():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1308_5426_gb300
    return paper_1308_5426_gb300


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_gpu_cumulants_match_exact_enumeration(plr, precision):
    from paper_1308_5426_gb300.analysis import observables
    L, q, sigma, c = 8, 3, 0.5, 2
    ratios = np.array([0.15, 0.3, 0.6])
    temps = ratios * oracle.jtot(L, sigma)
    j = plr.Job(L, q, sigma, temps, 2024, precision=precision, recompute_every=50, pair_factor=c)
    for _ in range(500):
        j.sweep(1)
        j.exchange()
    n = 40_000
    E = np.zeros((n, 3))
    M = np.zeros((n, 3))
    for k in range(n):
        j.sweep(1)
        j.exchange()
        E[k], M[k] = j.measure()
    j.close()
    got = observables(E, M, L, nblocks=40)
    ex = exact_averages(L, q, oracle.jstar(L, sigma), c, 1.0 / temps)
    ue_x = ex["E4"] / ex["E2"] ** 2
    vm_x = 1.0 - ex["M4"] / (3.0 * ex["M2"] ** 2)
    for t in range(3):
        assert abs(got["UE"][t] - ue_x[t]) < 3 * got["UE_err"][t] + 1e-6, (t, got["UE"][t], ue_x[t])
        assert abs(got["VM"][t] - vm_x[t]) < 3 * got["VM_err"][t] + 1e-6, (t, got["VM"][t], vm_x[t])
        assert abs(got["e"][t] - ex["E"][t] / L) < 3 * got["e_err"][t] + 1e-9
