"""The allocation-free measurement entry point (potts_lr_measure_static),
called through the C ABI with caller-owned device buffers, gives the same
energies and magnetisations as the handle's potts_lr_measure, on two calls in
a row with different configurations, and rejects sizes beyond its fixed
scratch; on a long chain (its shared memory above the 48 KB default) and with
pair factor 1 it matches the oracle's plain double sum.  This file is
collected last on purpose."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1308_5426_gb300 import workloads

pytestmark = pytest.mark.gpu


def _pack(S):
    """Packed spins [R][ceil(L/8)] uint32, spin i in bits 4(i%8) of word i/8."""
    R, L = S.shape
    W = (L + 7) // 8
    out = np.zeros((R, W), dtype=np.uint32)
    for i in range(L):
        out[:, i // 8] |= S[:, i].astype(np.uint32) << np.uint32(4 * (i % 8))
    return out


def test_measure_static_matches_measure():
    import __graft_entry__
    __graft_entry__.build()
    torch = pytest.importorskip("torch")
    import paper_1308_5426_gb300 as plr
    from paper_1308_5426_gb300 import _lib
    lib = _lib.load()
    L, q, sigma, R = 257, 5, 0.4, 6  # ragged L: a partial last word
    temps = workloads.geometric_ratios(R, 0.05, 1.0) * oracle.jtot(L, sigma)
    job = plr.Job(L, q, sigma, temps, 31)
    dev = torch.device("cuda", torch.cuda.current_device())
    J = torch.from_numpy(plr.jstar(L, sigma)).to(dev)
    stream = torch.cuda.current_stream(dev)
    for call in range(2):
        job.sweep(3)
        job.exchange()
        E_ref, M_ref = job.measure()
        spins = torch.from_numpy(_pack(job.spins()).view(np.int32)).to(dev)
        E = torch.full((R,), float("nan"), dtype=torch.float64, device=dev)
        M = torch.full((R,), float("nan"), dtype=torch.float64, device=dev)
        rc = lib.potts_lr_measure_static(ctypes.c_void_p(spins.data_ptr()), L, q, R,
                                         ctypes.c_void_p(J.data_ptr()), 2, ctypes.c_void_p(E.data_ptr()),
                                         ctypes.c_void_p(M.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert rc == _lib.OK, call
        torch.cuda.synchronize(dev)
        np.testing.assert_allclose(E.cpu().numpy(), E_ref, rtol=1e-10, err_msg="call %d" % call)
        np.testing.assert_allclose(M.cpu().numpy(), M_ref, rtol=0, atol=1e-14, err_msg="call %d" % call)
    # sizes beyond the fixed scratch are rejected before any device work
    big = 4097
    rc = lib.potts_lr_measure_static(ctypes.c_void_p(spins.data_ptr()), L, q, big, ctypes.c_void_p(J.data_ptr()),
                                     2, ctypes.c_void_p(E.data_ptr()), ctypes.c_void_p(M.data_ptr()), None)
    assert rc == _lib.EINVAL
    job.close()


def test_measure_static_long_chain_pair_once_against_oracle():
    """L = 25001 (a ragged last word; 7 distance tiles x 4 word tiles, so the
    tile sum of one slot spans many window loads) with c = 1: energies equal
    the oracle's plain O(L^2) double sum to 1e-10 and magnetisations to 1e-14,
    on two calls in a row."""
    import __graft_entry__
    __graft_entry__.build()
    torch = pytest.importorskip("torch")
    import paper_1308_5426_gb300 as plr
    from paper_1308_5426_gb300 import _lib
    lib = _lib.load()
    L, q, sigma, R = 25001, 3, 0.4, 2
    rng = np.random.default_rng(25001)
    S = rng.integers(0, q, size=(R, L)).astype(np.uint8)
    S[1, : 2 * L // 3] = 1  # an ordered stretch: energy and magnetisation far from the random ones
    o = oracle.Oracle(L, q, sigma, np.ones(R), 1, c=1, fields=False)
    o.set_spins(S)
    E_ref, M_ref = o.running_energy(), o.magnetisation()  # the plain double sum (Eq. 2), Eq. 10
    dev = torch.device("cuda", torch.cuda.current_device())
    J = torch.from_numpy(plr.jstar(L, sigma)).to(dev)
    spins = torch.from_numpy(_pack(S).view(np.int32)).to(dev)
    stream = torch.cuda.current_stream(dev)
    for call in range(2):
        E = torch.full((R,), float("nan"), dtype=torch.float64, device=dev)
        M = torch.full((R,), float("nan"), dtype=torch.float64, device=dev)
        rc = lib.potts_lr_measure_static(ctypes.c_void_p(spins.data_ptr()), L, q, R,
                                         ctypes.c_void_p(J.data_ptr()), 1, ctypes.c_void_p(E.data_ptr()),
                                         ctypes.c_void_p(M.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert rc == _lib.OK, call
        torch.cuda.synchronize(dev)
        np.testing.assert_allclose(E.cpu().numpy(), E_ref, rtol=1e-10, err_msg="call %d" % call)
        np.testing.assert_allclose(M.cpu().numpy(), M_ref, rtol=0, atol=1e-14, err_msg="call %d" % call)
