"""Host arithmetic of bench.py's roofline entries (no GPU): the algorithmic
work of one sweep launch over its measured duration, against the right
denominator for the kernel the library reports it ran (potts_lr_sweep_info):
FP64 or FP32 adds against the add pipe, FX64 update bytes against shared
memory where the fields sit there and against L2 where they sit in global
memory."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1308_5426_gb300 import workloads  # noqa: E402


class FakeLib:
    def __init__(self):
        self.asked = []

    def probe(self, what):
        self.asked.append(what)
        return {"smem": 4.0e13, "l2": 2.0e13, "fp64_add": 5.0e11, "fp32_add": 3.9e13, "i64_add": 1.0e13}[what]


def _info(kernel="memory", hs=True, js=True, rf=0, cl=0):
    return {"kernel": kernel, "fields_in_smem": hs, "table_in_smem": js, "register_config": rf, "cluster": cl,
            "threads": 256, "smem_bytes": 0}


def test_fx64_roofline_with_fields_in_shared_memory():
    specs = workloads.chains_jobs()
    for s in specs:
        s.precision = "fx64"
    lib = FakeLib()
    res = {"sweep_ms": [0.5, 0.5], "acceptance": 0.25, "info": _info()}
    r = bench.sweep_roofline(lib, res, specs, 2070.0, 152)
    att = 8 * 1024 * 64
    want = att * 0.25 * 1024 * 40 / 0.5e-3
    assert lib.asked == ["smem"]
    assert r["bound"] == "smem" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(want / 1e9)
    assert r["peak"] == pytest.approx(40000.0)
    assert r["frac"] == pytest.approx(want / 4.0e13)
    assert r["sweep_ms_avg"] == pytest.approx(0.5)
    assert "shared memory" in r["kernel"] and "long long" in r["kernel"]


def test_fx64_roofline_with_fields_in_global_memory_uses_l2():
    s = workloads.precision_job("fx64")
    lib = FakeLib()
    res = {"sweep_ms": [4.0], "acceptance": 0.1, "info": _info(hs=False, js=True)}
    r = bench.sweep_roofline(lib, res, [s], 2070.0, 152)
    want = 4096 * 128 * 0.1 * 4096 * 40 / 4e-3
    assert lib.asked == ["l2"] and r["bound"] == "l2"
    assert r["achieved"] == pytest.approx(want / 1e9)
    assert r["frac"] == pytest.approx(want / 2.0e13)
    assert "global memory" in r["kernel"]
    # 128 slots on 152 SMs: also against the occupied SMs
    assert r["occupied_sms"] == 128 and r["frac_of_occupied_sms"] == pytest.approx(r["frac"] * 152 / 128)


@pytest.mark.parametrize("prec,lanes", [("fp64", 2), ("fp32", 128)])
def test_alu_roofline(prec, lanes):
    specs = workloads.chains_jobs()
    for s in specs:
        s.precision = prec
    lib = FakeLib()
    info = _info("registers", rf=3) if prec == "fp32" else _info()
    res = {"sweep_ms": [0.6], "acceptance": 0.2, "info": info}
    r = bench.sweep_roofline(lib, res, specs, 2070.0, 152)
    adds = 8 * 1024 * 64 * 0.2 * 2 * 1024
    peak = 152 * lanes * 2070e6
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(adds / 0.6e-3 / 1e12)
    assert r["peak"] == pytest.approx(peak / 1e12)
    assert r["frac"] == pytest.approx(adds / 0.6e-3 / peak)
    assert "frac_of_occupied_sms" not in r  # 512 slots fill the SMs
    assert ("registers" in r["kernel"]) == (prec == "fp32")


def test_fx64_register_and_cluster_kernels():
    """FX64 fields in registers: 64-bit integer adds against the integer-add
    probe; FX64 fields shared by a cluster: shared-memory bytes."""
    specs = workloads.chains_jobs()
    for s in specs:
        s.precision = "fx64"
    lib = FakeLib()
    res = {"sweep_ms": [0.4], "acceptance": 0.2, "info": _info("registers", hs=False, js=False, rf=4)}
    r = bench.sweep_roofline(lib, res, specs, 2070.0, 152)
    adds = 8 * 1024 * 64 * 0.2 * 2 * 1024
    assert lib.asked == ["i64_add"] and r["bound"] == "alu"
    assert r["frac"] == pytest.approx(adds / 0.4e-3 / 1.0e13)
    assert "FX64 fields in registers" in r["kernel"]
    s = workloads.precision_job("fx64")
    lib = FakeLib()
    res = {"sweep_ms": [2.0], "acceptance": 0.14, "info": _info("cluster", hs=False, js=False, cl=2)}
    r = bench.sweep_roofline(lib, res, [s], 2070.0, 152)
    assert lib.asked == ["smem"] and r["bound"] == "smem"
    assert "FX64 fields shared by a 2-CTA cluster" in r["kernel"]
    assert "frac_of_occupied_sms" not in r
