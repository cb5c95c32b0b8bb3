"""Host arithmetic of bench.py's FX64 roofline entry (no GPU): the algorithmic
shared-memory bytes of the field updates over the measured launch time, against
a probe value, and the residency rule that decides whether that roofline
applies (the library keeps FX64 fields and table in shared memory while they
fit its 220 KB budget)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1308_5426_gb300 import workloads  # noqa: E402


class FakeLib:
    def probe(self, what):
        assert what == "smem"
        return 4.0e13


def test_fx64_roofline_on_the_chain_workload():
    specs = workloads.chains_jobs()
    res = {"sweep_ms": [0.5, 0.5], "acceptance": 0.25}
    r = bench.fx64_smem_roofline(FakeLib(), res, specs)
    att = 8 * 1024 * 64
    want = att * 0.25 * 1024 * 40 / 0.5e-3
    assert r["bound"] == "smem" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(want / 1e9)
    assert r["peak"] == pytest.approx(40000.0)
    assert r["frac"] == pytest.approx(want / 4.0e13)
    assert r["sweep_ms_avg"] == pytest.approx(0.5)


def test_fx64_residency_rule():
    # L = 1024, q = 5: 8.2 KB of table + 40 KB of fields: shared memory
    assert bench.fx64_fields_in_smem(1024, 5)
    # L = 4096, q = 8: 256 KB of fields: global memory
    assert not bench.fx64_fields_in_smem(4096, 8)
    # the boundary: q Lpad 8 + (Lpad + 4) 8 + the rest within 220 KB
    assert bench.fx64_fields_in_smem(2048, 12)
    assert not bench.fx64_fields_in_smem(2048, 13)
    s = workloads.precision_job("fx64")
    r = bench.fx64_smem_roofline(FakeLib(), {"sweep_ms": [4.0], "acceptance": 0.1}, [s])
    assert r["bound"] is None and "global" in r["kernel"]
