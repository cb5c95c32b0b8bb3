"""The C ABI library builds, loads and exports every entry point that
include/potts_lr.h declares; its host-side J* builder agrees with the oracle
(no GPU needed for either)."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1308_5426_gb300 import _lib, build
    build.build()
    return _lib.load()


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"^\s*(?:int|void|const char\*)\s+(potts_lr_\w+)\s*\(", src, re.M)
    return names


def test_exports_every_declared_symbol(lib):
    from paper_1308_5426_gb300 import _lib
    decl = _declared()
    assert len(decl) >= 20
    for name in decl:
        assert hasattr(lib, name), name
    assert sorted(decl) == sorted(_lib.EXPORTS)


def test_error_paths_without_gpu(lib):
    """Argument checks happen before any device work."""
    import ctypes
    from paper_1308_5426_gb300 import _lib
    h = ctypes.c_void_p()
    T = np.ones(4)
    bad = [(1, 3, 0.5), (64, 1, 0.5), (64, 17, 0.5), (64, 3, 0.0), (64, 3, float("nan"))]
    for L, q, s in bad:
        rc = lib.potts_lr_create(L, q, s, _lib._ptr(T), 4, 1, None, ctypes.byref(h))
        assert rc == _lib.EINVAL, (L, q, s)
        assert h.value is None
        assert len(lib.potts_lr_last_error()) > 0
    Tneg = np.array([1.0, -1.0])
    assert lib.potts_lr_create(64, 3, 0.5, _lib._ptr(Tneg), 2, 1, None, ctypes.byref(h)) == _lib.EINVAL
    assert lib.potts_lr_sweep(None, 1) == _lib.EINVAL
    assert lib.potts_lr_jstar(1, 0.5, None) == _lib.EINVAL


def test_option_checks_without_gpu(lib):
    """Unknown precisions and the kernel variants a precision cannot run are
    rejected before any device work (FX64 sweeps only on the shared/global
    memory kernel)."""
    import ctypes
    from paper_1308_5426_gb300 import _lib
    T = np.ones(4)
    bad = [dict(precision=3), dict(precision=-1),
           dict(precision=_lib.FX64, sweep_variant=4), dict(precision=_lib.FX64, site_order=1),
           dict(precision=_lib.FP32, sweep_variant=4), dict(precision=_lib.FP32, site_order=1),
           dict(pair_factor=3), dict(sweep_variant=6), dict(sweep_variant=25)]
    for kw in bad:
        o = _lib.Opts()
        assert lib.potts_lr_default_opts(ctypes.byref(o)) == _lib.OK
        for k, v in kw.items():
            setattr(o, k, v)
        h = ctypes.c_void_p()
        rc = lib.potts_lr_create(64, 3, 0.5, _lib._ptr(T), 4, 1, ctypes.byref(o), ctypes.byref(h))
        assert rc == _lib.EINVAL, kw
        assert h.value is None


def test_entry_point_argument_checks_without_gpu(lib):
    """NULL handles and out-of-range sizes are rejected before any device work:
    the batch calls, the allocation-free measurement (sizes beyond its fixed
    scratch included) and the probe."""
    import ctypes
    from paper_1308_5426_gb300 import _lib
    P = ctypes.c_void_p
    b = P()
    assert lib.potts_lr_batch_create(None, 1, None, ctypes.byref(b)) == _lib.EINVAL
    arr = (P * 2)(None, None)
    assert lib.potts_lr_batch_create(arr, 2, None, ctypes.byref(b)) == _lib.EINVAL
    assert lib.potts_lr_batch_create(arr, 0, None, ctypes.byref(b)) == _lib.EINVAL
    assert b.value is None
    assert lib.potts_lr_batch_run(None, 1, 1) == _lib.EINVAL
    assert lib.potts_lr_batch_sweep(None, 1) == _lib.EINVAL
    assert lib.potts_lr_batch_exchange(None) == _lib.EINVAL
    assert lib.potts_lr_batch_sync(None) == _lib.EINVAL
    n = ctypes.c_size_t()
    assert lib.potts_lr_batch_state_size(None, ctypes.byref(n)) == _lib.EINVAL
    assert lib.potts_lr_measure(None, None, None) == _lib.EINVAL
    assert lib.potts_lr_fields_recompute(None) == _lib.EINVAL
    assert lib.potts_lr_exchange(None) == _lib.EINVAL
    # potts_lr_measure_static(spins, L, q, R, jstar, pair_factor, E, M, stream):
    # the pointers are never dereferenced on these paths
    d = P(16)
    ok = dict(spins=d, L=64, q=3, R=4, jstar=d, c=2, E=d, M=d)
    for bad in (dict(spins=None), dict(jstar=None), dict(E=None), dict(M=None), dict(L=1), dict(q=1),
                dict(q=17), dict(R=0), dict(R=4097), dict(c=3)):
        a = dict(ok, **bad)
        rc = lib.potts_lr_measure_static(a["spins"], a["L"], a["q"], a["R"], a["jstar"], a["c"], a["E"], a["M"],
                                         None)
        assert rc == _lib.EINVAL, bad
    v = ctypes.c_double()
    assert lib.potts_lr_probe(5, ctypes.byref(v)) == _lib.EINVAL
    assert lib.potts_lr_probe(0, None) == _lib.EINVAL
    # the near-tie log, the wait limits and the sweep description of a NULL handle
    k = ctypes.c_int()
    ev = np.zeros((4, 5), np.int32)
    assert lib.potts_lr_near_log(None, _lib._ptr(ev), 4, ctypes.byref(k)) == _lib.EINVAL
    assert lib.potts_lr_set_wait_limits(None, 0, 0) == _lib.EINVAL
    info = np.zeros(7, np.int32)
    assert lib.potts_lr_sweep_info(None, _lib._ptr(info), 7) == _lib.EINVAL
    assert lib.potts_lr_set_rebuild_split(None, 2) == _lib.EINVAL
    assert lib.potts_lr_rebuild_info(None, None, None, None) == _lib.EINVAL


@pytest.mark.parametrize("L", [2, 3, 64, 1000, 1024, 4096, 16384, 65536])
@pytest.mark.parametrize("sigma", [0.01, 0.1, 0.2, 0.5, 1.0, 1.5, 3.0])
def test_jstar_builder_matches_oracle(lib, L, sigma):
    """Library J* (Euler-Maclaurin Hurwitz zeta, own code) vs the oracle's
    (scipy Hurwitz zeta) to 1e-14 relative, and exactly symmetric."""
    import oracle
    import paper_1308_5426_gb300 as plr
    J = plr.jstar(L, sigma)
    ref = oracle.jstar(L, sigma)
    assert J[0] == 0.0
    np.testing.assert_allclose(J[1:], ref[1:], rtol=1e-14, atol=0)
    r = np.arange(1, L)
    assert np.array_equal(J[r], J[L - r])
